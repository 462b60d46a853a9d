"""Packed (uneven) batches: one persistent launch per direction, each instance on the path
its own size selects; results must equal the same instance solved alone and the oracle."""
import numpy as np
import pytest
import torch

from paper_1703_00443_gb300 import inputs, qp_backward, qp_forward
from paper_1703_00443_gb300.packed import PackedBatch
from tests.helpers import grad_floor, oracle_many, rel_err, rel_err_inf

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
NAMES = ("dQ", "dq", "dG", "dh", "dA", "db")


def _instances(sizes, seed=0):
    return [inputs.random_qp(n, p, m, workload=inputs.WL_UNEVEN, index=i, seed=seed)
            for i, (n, p, m) in enumerate(sizes)]


def _grads_in(sizes, seed=0):
    return [inputs.upstream_grad(1, n, workload=inputs.WL_UNEVEN, start=i, seed=seed)[0]
            for i, (n, p, m) in enumerate(sizes)]


def _solve_packed(sizes, inst, gin, dtype=torch.float32, want_status=False):
    npdt = np.float32 if dtype == torch.float32 else np.float64
    pb = PackedBatch(sizes, dtype=dtype, device=DEV)
    Qp, qp, Gp, hp, Ap, bp = pb.pack([tuple(npdt(x) for x in t) for t in inst])
    out = pb.forward(Qp, qp, Gp, hp, Ap, bp)
    bst = torch.full((len(sizes),), -1, dtype=torch.int32, device=DEV)
    grads = pb.backward(Qp, Gp, Ap, pb.pack_vec([npdt(g) for g in gin], "q"), status=bst)
    torch.cuda.synchronize()
    res = dict(z=pb.unpack(out.z, "q"), lam=pb.unpack(out.lam, "h"), nu=pb.unpack(out.nu, "b"),
               status=out.status[: len(sizes)].cpu().numpy())
    for k, key, gbuf in zip(NAMES, pb.KEYS, grads):
        res[k] = pb.unpack(gbuf, key)
    if want_status:
        return pb, res, bst.cpu().numpy()
    return pb, res


def test_packed_equals_each_instance_alone():
    sizes = [(12, 9, 2), (100, 100, 50), (7, 13, 3), (140, 200, 30), (33, 40, 8), (64, 64, 16),
             (150, 90, 37)]
    inst = _instances(sizes, seed=5)
    gin = _grads_in(sizes, seed=5)
    pb, res = _solve_packed(sizes, inst, gin)
    assert pb.n_global >= 1 and pb.n_global < len(sizes)   # both kernel paths in one launch
    assert (res["status"] == 0).all()
    _assert_equal_alone(inst, gin, res, np.float32)


def _alone(t, g, npdt):
    """The instance solved alone: by qp_forward/qp_backward, or, for sizes whose fixed-size
    setup sweep takes the tensor cores (the packed kernels sweep on CUDA cores), as a packed
    batch of one."""
    from paper_1703_00443_gb300.qp import uses_tensor_cores
    n, p, m = t[0].shape[0], t[2].shape[0], t[4].shape[0]
    dtype = torch.float32 if npdt == np.float32 else torch.float64
    if uses_tensor_cores(dtype, n, p, m):
        _, r = _solve_packed([(n, p, m)], [t], [g], dtype=dtype)
        return {k: r[k][0] for k in ("z", "lam") + NAMES}
    T = [torch.from_numpy(npdt(x)).unsqueeze(0).to(DEV) for x in t]
    f = qp_forward(*T)
    gr = qp_backward(f, torch.from_numpy(npdt(g)).unsqueeze(0).to(DEV))
    torch.cuda.synchronize()
    out = {"z": f.z[0], "lam": f.lam[0]}
    out.update({k: gg[0] for k, gg in zip(NAMES, gr)})
    return out


def _assert_equal_alone(inst, gin, res, npdt):
    for i, t in enumerate(inst):
        a = _alone(t, gin[i], npdt)
        for k in ("z", "lam") + NAMES:
            assert torch.equal(a[k], res[k][i]), (i, k)


def test_packed_shared_memory_only_batch_equals_alone():
    """A batch with no global-path instance runs the packed kernel compiled with the
    shared-memory path alone; results stay those of each instance solved alone."""
    sizes = [(12, 9, 2), (100, 100, 50), (7, 13, 3), (33, 40, 8), (64, 64, 16), (5, 0, 2)]
    inst = _instances(sizes, seed=6)
    gin = _grads_in(sizes, seed=6)
    pb, res = _solve_packed(sizes, inst, gin)
    assert pb.n_global == 0
    assert (res["status"] == 0).all()
    _assert_equal_alone(inst, gin, res, np.float32)


def test_packed_fp64_mixed_paths_equals_alone():
    sizes = [(10, 20, 0), (30, 150, 5), (8, 12, 3), (40, 60, 10)]
    inst = _instances(sizes, seed=7)
    gin = _grads_in(sizes, seed=7)
    pb, res = _solve_packed(sizes, inst, gin, dtype=torch.float64)
    assert pb.n_global >= 1 and pb.n_global < len(sizes)
    assert (res["status"] == 0).all()
    _assert_equal_alone(inst, gin, res, np.float64)


def test_packed_uneven_sample_matches_oracle():
    """A sample of the uneven workload plus its largest shapes (n >= 200, and the
    (256, 512, 64) class that takes the global path's blocked factor): every result of every
    instance against the oracle, in both forms of the relative error; the backward status
    of every instance is CONVERGED."""
    sizes = inputs.uneven_sizes(24) + [(256, 512, 64), (230, 300, 40), (210, 105, 52)]
    inst = _instances(sizes)
    gin = _grads_in(sizes)
    pb, res, bst = _solve_packed(sizes, inst, gin, want_status=True)
    assert (res["status"] == 0).all(), res["status"]
    assert ((bst & 0xff) == 0).all(), bst
    assert pb.n_global >= 3
    refs = oracle_many([tuple(np.float64(x) for x in t) + (np.float64(np.float32(g)),)
                        for t, g in zip(inst, gin)])
    for i, g in enumerate(gin):
        sol, gr = refs[i]
        checks = [("z", sol["z"], 1e-5, None), ("lam", sol["lam"], 1e-4, None),
                  ("nu", sol["nu"], 1e-4, None)] + [(k, gr[k], 1e-4, k) for k in NAMES]
        for k, ref, tol, gname in checks:
            if ref.size == 0:
                continue
            x = res[k][i].double().cpu().numpy()[None]
            for fn, nrm in ((rel_err, 2), (rel_err_inf, np.inf)):
                fl = None if gname is None else grad_floor(gname, np.float32(g)[None],
                                                           sol["z"][None], norm=nrm)
                e = fn(x, ref[None], fl)[0]
                assert e <= tol, (i, sizes[i], k, nrm, e)


def test_packed_cuda_graph_replay_matches_eager():
    sizes = [(20, 30, 5), (90, 100, 20), (150, 120, 30), (40, 10, 0)]
    inst = _instances(sizes, seed=11)
    gin = _grads_in(sizes, seed=11)
    pb = PackedBatch(sizes, device=DEV)
    Qp, qp, Gp, hp, Ap, bp = pb.pack([tuple(np.float32(x) for x in t) for t in inst])
    gl = pb.pack_vec([np.float32(g) for g in gin], "q")
    eager = pb.forward(Qp, qp, Gp, hp, Ap, bp)
    eg = pb.backward(Qp, Gp, Ap, gl)
    torch.cuda.synchronize()
    ez, egrads = eager.z.clone(), [t.clone() for t in eg]
    # capture forward + backward with static buffers, then replay on the same data
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fout = pb.forward(Qp, qp, Gp, hp, Ap, bp)
        gout = pb.backward(Qp, Gp, Ap, gl)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        fout = pb.forward(Qp, qp, Gp, hp, Ap, bp, out=fout)
        gout = pb.backward(Qp, Gp, Ap, gl, out=gout)
    for _ in range(2):
        fout.z.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for a, b in zip(pb.unpack(fout.z, "q"), pb.unpack(ez, "q")):
            assert torch.equal(a, b)
        for key, a, b in zip(pb.KEYS, gout, egrads):
            for x, y in zip(pb.unpack(a, key), pb.unpack(b, key)):
                assert torch.equal(x, y), key


def test_autotuned_packed_batch_matches_alone_on_the_chosen_path():
    from paper_1703_00443_gb300 import autotune, default_options
    classes = [(16, 16, 4), (64, 64, 16), (96, 192, 0)]
    tun = autotune.autotune(device=DEV, classes=classes, save_to=None)
    sizes = [(16, 16, 4), (64, 64, 16), (96, 192, 0), (30, 20, 5)]
    inst = _instances(sizes, seed=21)
    gin = _grads_in(sizes, seed=21)
    hints, cost = tun.plan_arrays(sizes)
    assert (cost > 0).all()
    pb = PackedBatch(sizes, device=DEV, tuning=tun)
    Qp, qp, Gp, hp, Ap, bp = pb.pack([tuple(np.float32(x) for x in t) for t in inst])
    out = pb.forward(Qp, qp, Gp, hp, Ap, bp)
    torch.cuda.synchronize()
    zs = pb.unpack(out.z, "q")
    for i, t in enumerate(inst):
        o = default_options(torch.float32)
        o.path = 1 if hints[i] == 1 else 0
        T = [torch.from_numpy(np.float32(x)).unsqueeze(0).to(DEV) for x in t]
        f = qp_forward(*T, options=o)
        torch.cuda.synchronize()
        assert torch.equal(f.z[0], zs[i]), i
