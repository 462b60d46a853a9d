"""Serving loop on the GPU: mixed-size requests, continuous batching on several streams;
each request's result equals the same instance solved alone."""
import numpy as np
import pytest
import torch

from paper_1703_00443_gb300 import inputs, qp_backward, qp_forward
from paper_1703_00443_gb300.serving import QPServer, request_bytes

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
    T = [torch.from_numpy(x).unsqueeze(0).to(DEV) for x in data]
    f = qp_forward(*T)
    gr = qp_backward(f, torch.from_numpy(g).unsqueeze(0).to(DEV))
    torch.cuda.synchronize()
    out = {"z": f.z[0].cpu().numpy(), "lam": f.lam[0].cpu().numpy(), "nu": f.nu[0].cpu().numpy()}
    for k, t in zip(NAMES, gr):
        out[k] = t[0].cpu().numpy()
    return out


def test_served_results_equal_alone_and_batches_overlap():
    sizes = inputs.serve_sizes(40, n_hi=256)
    pool = _pool(sizes)
    server = QPServer(device=DEV, max_inflight=3, max_batch=8)
    try:
        futs = [server.submit(*data, g) for data, g in pool]
        results = [f.result(timeout=120) for f in futs]
    finally:
        server.close()
    st = server.stats()
    assert st["completed"] == len(pool) and st["batches"] >= 5   # batch cap forces several
    for (data, g), res in zip(pool, results):
        assert res["status"] == 0
        ref = _alone(data, g)
        for k in ref:
            assert np.array_equal(res[k], ref[k]), k


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
