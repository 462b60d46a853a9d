"""Serving loop on the GPU: mixed-size requests, continuous batching on several streams;
each request's result equals the same instance solved alone and matches the FP64 oracle."""
import numpy as np
import pytest
import torch

from paper_1703_00443_gb300 import inputs, qp_backward, qp_forward
from paper_1703_00443_gb300.serving import QPServer, request_bytes
from tests.helpers import oracle_many, rel_err, rel_err_inf

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
NAMES = ("dQ", "dq", "dG", "dh", "dA", "db")


def _pool(sizes, seed=3):
    pool = []
    for i, (n, p, m) in enumerate(sizes):
        data = inputs.random_qp(n, p, m, workload=inputs.WL_SERVE, index=i, seed=seed)
        g = inputs.upstream_grad(1, n, workload=inputs.WL_SERVE, start=i, seed=seed)[0]
        pool.append((tuple(np.float32(x) for x in data), np.float32(g)))
    return pool


def _alone(data, g):
    """The request solved alone: by qp_forward/qp_backward, or, for sizes whose fixed-size
    setup sweep takes the tensor cores (the server's packed kernels sweep on CUDA cores), as a
    packed batch of one."""
    from paper_1703_00443_gb300.packed import PackedBatch
    from paper_1703_00443_gb300.qp import uses_tensor_cores
    n, p, m = data[0].shape[0], data[2].shape[0], data[4].shape[0]
    if uses_tensor_cores(torch.float32, n, p, m):
        pb = PackedBatch([(n, p, m)], device=DEV)
        P = pb.pack([data])
        fo = pb.forward(*P)
        go = pb.backward(P[0], P[2], P[4], pb.pack_vec([g], "q"))
        torch.cuda.synchronize()
        out = {"z": pb.unpack(fo.z, "q")[0], "lam": pb.unpack(fo.lam, "h")[0],
               "nu": pb.unpack(fo.nu, "b")[0]}
        for k, key, t in zip(NAMES, pb.KEYS, go):
            out[k] = pb.unpack(t, key)[0]
        return {k: v.cpu().numpy() for k, v in out.items()}
    T = [torch.from_numpy(x).unsqueeze(0).to(DEV) for x in data]
    f = qp_forward(*T)
    gr = qp_backward(f, torch.from_numpy(g).unsqueeze(0).to(DEV))
    torch.cuda.synchronize()
    out = {"z": f.z[0].cpu().numpy(), "lam": f.lam[0].cpu().numpy(), "nu": f.nu[0].cpu().numpy()}
    for k, t in zip(NAMES, gr):
        out[k] = t[0].cpu().numpy()
    return out


def test_served_results_equal_alone_match_oracle_and_batches_overlap():
    # mixed sizes, including instances on the global-memory kernel path (n >= 200)
    sizes = inputs.serve_sizes(40, n_hi=256) + [(200, 200, 50), (256, 256, 64), (230, 230, 57)]
    pool = _pool(sizes)
    server = QPServer(device=DEV, max_inflight=3, max_batch=8)
    try:
        futs = [server.submit(*data, g) for data, g in pool]
        results = [f.result(timeout=300) for f in futs]
        server.equalize_staging()
        n_in, n_out, nb = server.stage_peak
        assert n_in > 0 and all(st.inp.numel() >= n_in and st.out.numel() >= n_out
                                for st in server.staging)
    finally:
        server.close()
    st = server.stats()
    assert st["completed"] == len(pool) and st["batches"] >= 5   # batch cap forces several
    assert st["max_inflight_seen"] >= 2          # a batch was launched while another ran
    refs = oracle_many([tuple(np.float64(x) for x in data) + (np.float64(g),) for data, g in pool])
    for i, ((data, g), res) in enumerate(zip(pool, results)):
        assert res["status"] == 0
        alone = _alone(data, g)
        for k in alone:
            assert np.array_equal(res[k], alone[k]), k
        sol, gr = refs[i]
        gn = np.linalg.norm(np.float64(g))
        for k, ref, tol in (("z", sol["z"], 1e-5), ("lam", sol["lam"], 1e-4),
                            ("nu", sol["nu"], 1e-4)) + tuple((k, gr[k], 1e-4) for k in NAMES):
            if ref.size == 0:
                continue
            fl = 1e-12
            if k.startswith("d"):
                fl = 1e-3 * gn * (max(1.0, np.linalg.norm(sol["z"])) if k in ("dQ", "dG", "dA") else 1.0)
            x = np.float64(res[k]).reshape(1, -1)
            e2 = rel_err(x, ref.reshape(1, -1), fl)[0]
            ei = rel_err_inf(x, ref.reshape(1, -1), fl)[0]
            assert e2 <= tol and ei <= tol, (i, sizes[i], k, e2, ei)


def test_hbm_budget_admission_and_rejection():
    sizes = [(20, 20, 5)] * 6 + [(200, 200, 50)]
    pool = _pool(sizes, seed=4)
    small = request_bytes((20, 20, 5))
    server = QPServer(device=DEV, max_inflight=2, max_batch=64, hbm_budget_bytes=3 * small)
    try:
        futs = [server.submit(*data, g) for data, g in pool]
        done = [f.exception(timeout=120) is None for f in futs]
    finally:
        server.close()
    assert done[:6] == [True] * 6
    assert isinstance(futs[6].exception(), MemoryError)   # larger than the whole budget
    assert server.stats()["batches"] >= 2                  # at most 3 requests per admission
