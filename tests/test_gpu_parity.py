"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded inputs.

Tolerances: FP32 path z* rel err ≤ 1e-5 and every gradient rel err ≤ 1e-4 (per instance,
‖x − x_ref‖₂/‖x_ref‖₂); FP64 path ≤ 1e-9 on z*, λ*, ν* and ≤ 1e-8 on gradients.
"""
import numpy as np
import pytest
import torch

from paper_1703_00443_gb300 import inputs, qp_backward, qp_forward, supported
from tests.helpers import (grad_floor, kkt_residuals_fp64, oracle_solve_and_grad, rel_err,
                           rel_err_inf)

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GRAD_NAMES = ("dQ", "dq", "dG", "dh", "dA", "db")


def _to_dev(batch, dtype):
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    return [torch.from_numpy(np.ascontiguousarray(x)).to(DEV, tdt) for x in
            (batch.Q, batch.q, batch.G, batch.h, batch.A, batch.b)]


def _run(batch, g, dtype):
    T = _to_dev(batch, dtype)
    fwd = qp_forward(*T)
    grads = qp_backward(fwd, torch.from_numpy(np.ascontiguousarray(g)).to(T[0].device, T[0].dtype))
    torch.cuda.synchronize()
    out = dict(z=fwd.z.cpu().double().numpy(), lam=fwd.lam.cpu().double().numpy(),
               nu=fwd.nu.cpu().double().numpy(), status=fwd.status.cpu().numpy(),
               iters=fwd.iters.cpu().numpy())
    for k, v in zip(GRAD_NAMES, grads):
        out[k] = v.cpu().double().numpy()
    return out


def _compare(batch, g, out, idx, ztol, gtol, ltol=None):
    """Oracle parity of the selected instances in both forms of the relative error: per
    instance ‖x − x_ref‖₂/max(‖x_ref‖₂, floor) and max_i |x_i − x_ref,i|/max(‖x_ref‖∞, floor).
    Returns the worst value of each result in each form."""
    idx = list(idx)
    sols, grads = oracle_solve_and_grad(batch, g, idx)
    worst = {}
    for name, ref_of, tol in (("z", lambda s, gr: s["z"], ztol),
                              ("lam", lambda s, gr: s["lam"], ltol),
                              ("nu", lambda s, gr: s["nu"], ltol)):
        ref = [ref_of(s, None) for s in sols]
        if tol is None or np.asarray(ref).size == 0:
            continue
        for form, fn in (("l2", rel_err), ("inf", rel_err_inf)):
            e = fn(out[name][idx], ref)
            worst[(name, form)] = e.max()
            assert e.max() <= tol, (name, form, e.max(), idx[int(np.argmax(e))])
    gsel = np.asarray(g)[idx]
    zref = [s["z"] for s in sols]
    for k in GRAD_NAMES:
        ref = [gr[k] for gr in grads]
        if np.asarray(ref).size == 0:
            continue
        for form, fn, nrm in (("l2", rel_err, 2), ("inf", rel_err_inf, np.inf)):
            e = fn(out[k][idx], ref, grad_floor(k, gsel, zref, norm=nrm))
            worst[(k, form)] = e.max()
            assert e.max() <= gtol, (k, form, e.max(), idx[int(np.argmax(e))])
    return worst


def test_plain_fp64_config():
    """Plain method in FP64: 8 QPs, n = 10, 20 inequalities, no equalities."""
    batch = inputs.random_batch(8, 10, 20, 0, workload=inputs.WL_PLAIN, dtype=np.float64)
    g = inputs.upstream_grad(8, 10, workload=inputs.WL_PLAIN, dtype=np.float64)
    out = _run(batch, g, np.float64)
    assert (out["status"] == 0).all()
    _compare(batch, g, out, range(8), 1e-9, 1e-8, ltol=1e-8)


@pytest.mark.parametrize("n", [10, 50, 100])
def test_sweep_fp32(n):
    """Timing-sweep shapes (n, nineq = n, neq = n/2), FP32 with FP64 residuals."""
    B = 8
    batch = inputs.random_batch(B, n, n, n // 2, workload=inputs.WL_SWEEP, dtype=np.float32)
    g = inputs.upstream_grad(B, n, workload=inputs.WL_SWEEP)
    out = _run(batch, g, np.float32)
    assert (out["status"] == 0).all(), out["status"]
    _compare(batch, g, out, range(B), 1e-5, 1e-4, ltol=1e-4)


def test_full_batch_oracle_parity_and_certified():
    """The benchmark launch (B = 128, n = 100, 100 inequalities, 50 equalities): every
    instance passes an FP64 KKT certificate and matches the oracle on z*, λ*, ν* and all six
    gradients, in the 2-norm and the ∞-norm forms of the relative error."""
    B, n = 128, 100
    batch = inputs.random_batch(B, n, n, n // 2, workload=inputs.WL_SWEEP, dtype=np.float32)
    g = inputs.upstream_grad(B, n, workload=inputs.WL_SWEEP)
    out = _run(batch, g, np.float32)
    assert (out["status"] == 0).all()
    cert = kkt_residuals_fp64(batch, out["z"], out["lam"], out["nu"])
    # z*, λ*, ν* are rounded to FP32 on output, which bounds what the certificate can show.
    assert cert[:, 0].max() <= 1e-4 and cert[:, 1].max() <= 1e-5
    assert cert[:, 2].max() <= 1e-5 and cert[:, 3].max() <= 0
    worst = _compare(batch, g, out, range(B), 1e-5, 1e-4, ltol=1e-4)
    print("worst relative errors over the 128 instances:",
          {f"{k}/{f}": f"{v:.2e}" for (k, f), v in worst.items()})


def test_onehot_structured():
    """Structured one-hot QP: Q = 0.1 I, z ≥ 0, 40 dense equalities, MSE-loss gradient."""
    B, n, neq = 16, 64, 40
    batch = inputs.onehot_batch(B, n, neq, dtype=np.float32)
    target = inputs.onehot_target(B, n)
    T = _to_dev(batch, np.float32)
    fwd = qp_forward(*T)
    torch.cuda.synchronize()
    z = fwd.z.cpu().double().numpy()
    g = (2.0 / n) * (z - target)
    out = _run(batch, g, np.float32)
    assert (out["status"] == 0).all()
    _compare(batch, g.astype(np.float32), out, range(B), 1e-5, 1e-4)


@pytest.mark.parametrize("n,nineq,neq", [(7, 13, 3), (1, 2, 0), (5, 0, 2), (12, 0, 0),
                                         (33, 9, 0), (60, 170, 10), (3, 1, 1),
                                         (135, 109, 8), (87, 157, 8)])
def test_ragged_and_edge_sizes(n, nineq, neq):
    B = 5
    assert supported(torch.float32, n, nineq, neq)
    batch = inputs.random_batch(B, n, nineq, neq, workload=inputs.WL_PLAIN, dtype=np.float32,
                                start=1000)
    g = inputs.upstream_grad(B, n, workload=inputs.WL_PLAIN, start=1000)
    out = _run(batch, g, np.float32)
    assert (out["status"] == 0).all(), out["status"]
    _compare(batch, g, out, range(B), 1e-5, 1e-4)


def test_empty_batch_is_noop():
    T = [torch.empty((0, 4, 4), device=DEV), torch.empty((0, 4), device=DEV),
         torch.empty((0, 3, 4), device=DEV), torch.empty((0, 3), device=DEV), None, None]
    fwd = qp_forward(*T)
    grads = qp_backward(fwd, torch.empty((0, 4), device=DEV))
    assert fwd.z.shape == (0, 4) and grads[0].shape == (0, 4, 4)


def test_indefinite_q_reports_not_pd():
    batch = inputs.random_batch(3, 6, 8, 2, workload=inputs.WL_PLAIN, dtype=np.float32)
    batch.Q[1] = -batch.Q[1]
    T = _to_dev(batch, np.float32)
    fwd = qp_forward(*T)
    grads = qp_backward(fwd, torch.ones((3, 6), device=DEV))
    torch.cuda.synchronize()
    st = fwd.status.cpu().numpy()
    assert st[0] == 0 and st[1] == 2 and st[2] == 0
    assert torch.isnan(fwd.z[1]).all() and torch.isnan(grads[0][1]).all()
    assert torch.isfinite(fwd.z[0]).all() and torch.isfinite(grads[0][2]).all()


def test_instance_alone_equals_in_batch_and_deterministic():
    batch = inputs.random_batch(16, 30, 30, 15, workload=inputs.WL_SWEEP, dtype=np.float32)
    g = inputs.upstream_grad(16, 30)
    full = _run(batch, g, np.float32)
    again = _run(batch, g, np.float32)
    one = inputs.random_batch(1, 30, 30, 15, workload=inputs.WL_SWEEP, dtype=np.float32, start=9)
    alone = _run(one, g[9:10], np.float32)
    for k in ("z", "lam", "nu") + GRAD_NAMES:
        assert np.array_equal(full[k], again[k]), k
        assert np.array_equal(full[k][9:10], alone[k]), k


def _run_opts(batch, g, dtype, options):
    T = _to_dev(batch, dtype)
    fwd = qp_forward(*T, options=options)
    grads = qp_backward(fwd, torch.from_numpy(np.ascontiguousarray(g)).to(T[0].device, T[0].dtype))
    torch.cuda.synchronize()
    out = dict(z=fwd.z.cpu().double().numpy(), lam=fwd.lam.cpu().double().numpy(),
               nu=fwd.nu.cpu().double().numpy(), status=fwd.status.cpu().numpy())
    for k, v in zip(GRAD_NAMES, grads):
        out[k] = v.cpu().double().numpy()
    return out


@pytest.mark.parametrize("n,nineq,neq", [(7, 13, 3), (33, 9, 0), (12, 0, 5), (50, 50, 25),
                                         (20, 37, 19)])
def test_global_memory_kernel_small_sizes(n, nineq, neq):
    """The global-memory kernel (forced) on sizes the oracle checks quickly, including
    padding of n + neq to the 16-pivot blocks and a partial last Cholesky block."""
    from paper_1703_00443_gb300 import default_options
    opts = default_options(torch.float32)
    opts.path = 1
    B = 4
    batch = inputs.random_batch(B, n, nineq, neq, workload=inputs.WL_PLAIN, dtype=np.float32,
                                start=2000)
    g = inputs.upstream_grad(B, n, workload=inputs.WL_PLAIN, start=2000)
    out = _run_opts(batch, g, np.float32, opts)
    assert (out["status"] == 0).all(), out["status"]
    _compare(batch, g, out, range(B), 1e-5, 1e-4, ltol=1e-4)


@pytest.mark.parametrize("dtype,path,n,nineq,neq", [(np.float32, 0, 20, 30, 5),
                                                    (np.float32, 1, 16, 181, 4),
                                                    (np.float64, 0, 10, 20, 3)])
def test_gradients_through_lambda_and_nu(dtype, path, n, nineq, neq):
    """ℓ = g_zᵀz* + g_λᵀλ* + g_νᵀν* through qp_backward_ext: the adjoint with the extra
    right-hand-side blocks, against the oracle (shared-memory path, the global path's blocked
    factor, FP64)."""
    from paper_1703_00443_gb300 import default_options
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    opts = default_options(tdt)
    opts.path = path
    B = 3
    batch = inputs.random_batch(B, n, nineq, neq, workload=inputs.WL_PLAIN, dtype=dtype, start=900)
    r = np.random.default_rng(9)
    gz = r.standard_normal((B, n)).astype(dtype)
    gl = r.standard_normal((B, nineq)).astype(dtype)
    gn = r.standard_normal((B, neq)).astype(dtype)
    T = _to_dev(batch, dtype)
    fwd = qp_forward(*T, options=opts)
    grads = qp_backward(fwd, torch.from_numpy(gz).to(DEV), dl_dlam=torch.from_numpy(gl).to(DEV),
                        dl_dnu=torch.from_numpy(gn).to(DEV))
    torch.cuda.synchronize()
    assert (fwd.status == 0).all()
    import oracle
    tol = 1e-4 if dtype == np.float32 else 1e-8
    for i in range(B):
        Q, q, G, h, A, b = batch.instance(i)
        sol = oracle.solve(Q, q, G, h, A, b)
        ref = oracle.backward(Q, G, h, A, sol, gz[i].astype(np.float64), gl[i].astype(np.float64),
                              gn[i].astype(np.float64))
        scale = np.linalg.norm(np.concatenate([gz[i], gl[i], gn[i]]).astype(np.float64))
        for k, t in zip(GRAD_NAMES, grads):
            got = t[i].double().cpu().numpy()
            if ref[k].size == 0:
                continue
            fl = 1e-3 * scale * (max(1.0, np.linalg.norm(sol["z"])) if k in ("dQ", "dG", "dA") else 1.0)
            e = np.linalg.norm(got - ref[k]) / max(np.linalg.norm(ref[k]), fl)
            assert e <= tol, (i, k, e)


def test_nearly_degenerate_instance_gradients_fp32():
    """An instance of the n = 50 timing sweep whose most weakly resolved constraint has
    max(λ_i, s_i) ≈ 5e-4 at the solution.  Its gradient is sensitive to how far the final
    iterate resolves that pair (s_i/λ_i enters the system the backward pass solves), so the
    FP32 path's stopping test also requires resolved complementarity pairs."""
    B, n = 1, 50
    batch = inputs.random_batch(B, n, n, n // 2, workload=inputs.WL_SWEEP, dtype=np.float32,
                                start=16)
    g = inputs.upstream_grad(B, n, workload=inputs.WL_SWEEP, start=16)
    sols, _ = oracle_solve_and_grad(batch, g, range(B))
    slack = batch.h[0] - batch.G[0] @ sols[0]["z"]
    assert np.min(np.maximum(sols[0]["lam"], slack)) < 1e-3     # the premise: nearly degenerate
    out = _run(batch, g, np.float32)
    assert (out["status"] == 0).all(), out["status"]
    _compare(batch, g, out, range(B), 1e-5, 1e-4, ltol=1e-4)


@pytest.mark.parametrize("n,nineq,neq", [(60, 203, 10), (40, 180, 0), (24, 177, 7)])
def test_global_memory_blocked_cholesky_fp32(n, nineq, neq):
    """The global-memory kernel (forced) where the Schur complement is too large for the
    register-tile Cholesky (nineq > 176): blocked factor with block-substitution solves,
    including nineq not a multiple of 4 (unaligned rows of the factor) and of the block."""
    from paper_1703_00443_gb300 import default_options
    opts = default_options(torch.float32)
    opts.path = 1
    B = 2
    batch = inputs.random_batch(B, n, nineq, neq, workload=inputs.WL_PLAIN, dtype=np.float32,
                                start=3000)
    g = inputs.upstream_grad(B, n, workload=inputs.WL_PLAIN, start=3000)
    out = _run_opts(batch, g, np.float32, opts)
    assert (out["status"] == 0).all(), out["status"]
    _compare(batch, g, out, range(B), 1e-5, 1e-4, ltol=1e-4)


@pytest.mark.parametrize("n,nineq,neq", [(20, 40, 4), (30, 150, 5)])
def test_global_memory_kernel_fp64(n, nineq, neq):
    """The global-memory kernel (forced) in FP64: the register-tile Cholesky (nineq = 40) and
    the blocked factor with 16-wide blocks (nineq = 150), at the FP64 tolerances."""
    from paper_1703_00443_gb300 import default_options
    opts = default_options(torch.float64)
    opts.path = 1
    B = 2
    batch = inputs.random_batch(B, n, nineq, neq, workload=inputs.WL_PLAIN, dtype=np.float64,
                                start=4000)
    g = inputs.upstream_grad(B, n, workload=inputs.WL_PLAIN, dtype=np.float64, start=4000)
    out = _run_opts(batch, g, np.float64, opts)
    assert (out["status"] == 0).all(), out["status"]
    _compare(batch, g, out, range(B), 1e-9, 1e-8, ltol=1e-8)


@pytest.mark.parametrize("n,nineq,neq", [(500, 500, 250), (256, 512, 64)])
def test_global_memory_kernel_large_sizes(n, nineq, neq):
    """Sizes whose factors exceed shared memory: the timing sweep's n = 500 point and the
    largest instance shape of the uneven workload."""
    from paper_1703_00443_gb300.qp import uses_global_path
    assert uses_global_path(torch.float32, n, nineq, neq)
    B = 2
    batch = inputs.random_batch(B, n, nineq, neq, workload=inputs.WL_SWEEP, dtype=np.float32)
    g = inputs.upstream_grad(B, n, workload=inputs.WL_SWEEP)
    out = _run(batch, g, np.float32)
    assert (out["status"] == 0).all(), out["status"]
    _compare(batch, g, out, range(B), 1e-5, 1e-4, ltol=1e-4)


@pytest.mark.parametrize("n,nineq,neq,path", [(100, 60, 44, 1), (100, 100, 50, 1), (96, 37, 32, 1),
                                              (140, 200, 30, 0), (150, 90, 37, 0),
                                              (180, 70, 60, 1), (150, 0, 40, 1),
                                              (160, 100, 0, 1), (200, 201, 17, 0)])
def test_tensor_core_setup_sweep(n, nineq, neq, path):
    """FP32 sizes whose fixed-size setup sweep takes its rank-64 updates on the tensor cores
    (tcgen05): 2–4 superblocks, the last one partial with 16, 32 or 48 pivots or whole,
    λ blocks of 0, 37, 90 (not multiples of 4), 200 and 201 rows (two λ tiles), no equality
    constraints, a
    Schur complement past the register-tile Cholesky (nineq > 176), against the oracle."""
    from paper_1703_00443_gb300 import default_options
    from paper_1703_00443_gb300.qp import uses_tensor_cores
    opts = default_options(torch.float32)
    opts.path = path
    assert uses_tensor_cores(torch.float32, n, nineq, neq, options=opts)
    B = 3
    batch = inputs.random_batch(B, n, nineq, neq, workload=inputs.WL_PLAIN, dtype=np.float32,
                                start=6000)
    g = inputs.upstream_grad(B, n, workload=inputs.WL_PLAIN, start=6000)
    out = _run_opts(batch, g, np.float32, opts)
    assert (out["status"] == 0).all(), out["status"]
    _compare(batch, g, out, range(B), 1e-5, 1e-4, ltol=1e-4)
