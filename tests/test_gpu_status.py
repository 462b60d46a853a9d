"""Per-instance statuses and the workspace stamp, each forced from the host:
max_iter reached, a non-finite input, infeasible data (with its Farkas certificate checked in
FP64 here), the time limit, a nearly degenerate solution, and a backward pass given a
workspace that holds no matching forward pass."""
import numpy as np
import pytest
import torch

from paper_1703_00443_gb300 import (FLAG_NEAR_DEGENERATE, STATUS_CONVERGED, STATUS_INFEASIBLE,
                                    STATUS_MAX_ITER, STATUS_NO_FORWARD, STATUS_NUMERICAL,
                                    STATUS_TIMEOUT, default_options, inputs, qp_backward,
                                    qp_forward)
from paper_1703_00443_gb300.qp import alloc_workspace

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _dev(batch, dt=torch.float32):
    return [torch.from_numpy(np.ascontiguousarray(x)).to(DEV, dt) for x in
            (batch.Q, batch.q, batch.G, batch.h, batch.A, batch.b)]


def _bwd(fwd, g, **kw):
    B = fwd.z.shape[0]
    st = torch.full((B,), -1, dtype=torch.int32, device=DEV)
    grads = qp_backward(fwd, g, status=st, **kw)
    torch.cuda.synchronize()
    return grads, st.cpu().numpy()


def test_max_iter_returns_finite_iterate_and_gradients():
    batch = inputs.random_batch(6, 30, 30, 15, workload=inputs.WL_SWEEP, start=40)
    opts = default_options(torch.float32)
    opts.max_iter = 2
    fwd = qp_forward(*_dev(batch), options=opts)
    g = torch.ones((6, 30), device=DEV)
    grads, bst = _bwd(fwd, g)
    assert (fwd.status.cpu().numpy() == STATUS_MAX_ITER).all()
    assert (fwd.iters.cpu().numpy() == 2).all()
    assert torch.isfinite(fwd.z).all() and torch.isfinite(fwd.lam).all()
    assert ((bst & 0xff) == STATUS_MAX_ITER).all()
    assert all(torch.isfinite(t).all() for t in grads)


def test_non_finite_input_gives_numerical_status_only_there():
    batch = inputs.random_batch(4, 12, 20, 3, workload=inputs.WL_PLAIN, start=70)
    batch.q[1, 3] = np.nan
    fwd = qp_forward(*_dev(batch))
    grads, bst = _bwd(fwd, torch.ones((4, 12), device=DEV))
    st = fwd.status.cpu().numpy()
    assert st[1] == STATUS_NUMERICAL and (st[[0, 2, 3]] == STATUS_CONVERGED).all()
    assert torch.isnan(fwd.z[1]).all() and torch.isfinite(fwd.z[[0, 2, 3]]).all()
    assert bst[1] == STATUS_NUMERICAL and ((bst[[0, 2, 3]] & 0xff) == 0).all()
    assert all(torch.isnan(t[1]).all() for t in grads)
    assert all(torch.isfinite(t[[0, 2, 3]]).all() for t in grads)


def _infeasible_batch(dtype):
    """Instance 0: z ≤ −1 and z ≥ 1 (G = [I; −I], h = −1).  Instance 1: z_1 + z_2 = 10 with
    every z_i ≤ 1 and ≥ −1.  Instance 2: a strictly feasible QP of the same sizes."""
    n = 4
    rng = np.random.default_rng(11)
    Q = np.stack([np.eye(n)] * 3)
    q = rng.standard_normal((3, n))
    G = np.stack([np.vstack([np.eye(n), -np.eye(n)])] * 3)
    h = np.stack([-np.ones(2 * n), np.ones(2 * n), 2.0 * np.ones(2 * n)])
    A = np.zeros((3, 1, n))
    A[:, 0, :2] = 1.0
    b = np.array([[0.0], [10.0], [0.5]])
    return inputs.QPBatch(Q, q, G, h, A, b).astype(dtype)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_infeasible_data_returns_a_farkas_certificate(dtype):
    batch = _infeasible_batch(dtype)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    fwd = qp_forward(*_dev(batch, tdt))
    grads, bst = _bwd(fwd, torch.ones((3, 4), device=DEV, dtype=tdt))
    st = fwd.status.cpu().numpy()
    assert st[2] == STATUS_CONVERGED, st
    assert (st[:2] == STATUS_INFEASIBLE).all(), st
    lam = fwd.lam.cpu().double().numpy()
    nu = fwd.nu.cpu().double().numpy()
    z = fwd.z.cpu().double().numpy()
    for i in range(2):
        Q, q, G, h, A, b = batch.instance(i)
        assert (lam[i] >= 0).all() and np.isfinite(z[i]).all()
        assert max(np.abs(lam[i]).max(), np.abs(nu[i]).max()) == pytest.approx(1.0, rel=1e-6)
        gap = -(h @ lam[i] + b @ nu[i])
        w = G.T @ lam[i] + A.T @ nu[i]
        # Farkas: (Gᵀλ + Aᵀν)ᵀz' ≤ hᵀλ + bᵀν for every feasible z', so a feasible point would
        # need ‖z'‖∞ ≥ gap/‖w‖₁; the kernel certifies 1e3·(1 + ‖z‖∞) before rounding its output
        bound = gap / np.abs(w).sum()
        assert gap > 0 and bound >= 1e2 * (1 + np.abs(z[i]).max()), (i, gap, bound)
    assert bst[0] == STATUS_INFEASIBLE and bst[1] == STATUS_INFEASIBLE
    assert all(torch.isnan(t[:2]).all() for t in grads if t.shape[1] > 0)


def test_time_limit_stops_with_timeout_and_usable_iterate():
    batch = inputs.random_batch(4, 60, 60, 30, workload=inputs.WL_SWEEP, start=90)
    opts = default_options(torch.float32)
    opts.time_limit_us = 1
    fwd = qp_forward(*_dev(batch), options=opts)
    grads, bst = _bwd(fwd, torch.ones((4, 60), device=DEV))
    st = fwd.status.cpu().numpy()
    assert (st == STATUS_TIMEOUT).all(), st
    assert (fwd.iters.cpu().numpy() <= 2).all()
    assert torch.isfinite(fwd.z).all()
    assert ((bst & 0xff) == STATUS_TIMEOUT).all()
    assert all(torch.isfinite(t).all() for t in grads)
    opts.time_limit_us = 10_000_000          # generous: converges as without a limit
    ref = qp_forward(*_dev(batch))
    lim = qp_forward(*_dev(batch), options=opts)
    torch.cuda.synchronize()
    assert (lim.status == 0).all() and torch.equal(lim.z, ref.z)


def test_near_degenerate_solution_is_flagged_in_the_backward_status():
    """A constraint through the unconstrained minimiser, z_u = −Q⁻¹q, is active with λ* = 0:
    both members of its complementarity pair vanish at the solution."""
    n, p = 5, 4
    rng = np.random.default_rng(5)
    Q = np.eye(n)[None].repeat(2, 0)
    q = rng.standard_normal((2, n))
    G = rng.standard_normal((2, p, n))
    zu = -q
    h = np.einsum("bij,bj->bi", G, zu) + 1.0
    h[0, 0] = G[0, 0] @ zu[0]          # instance 0: degenerate constraint 0
    batch = inputs.QPBatch(Q, q, G, h, np.zeros((2, 0, n)), np.zeros((2, 0))).astype(np.float64)
    fwd = qp_forward(*_dev(batch, torch.float64))
    _, bst = _bwd(fwd, torch.ones((2, n), device=DEV, dtype=torch.float64))
    assert (fwd.status.cpu().numpy() == STATUS_CONVERGED).all()
    assert (bst & 0xff == STATUS_CONVERGED).all()
    assert bst[0] & FLAG_NEAR_DEGENERATE and not bst[1] & FLAG_NEAR_DEGENERATE


def test_backward_rejects_a_workspace_without_matching_forward():
    batch = inputs.random_batch(3, 10, 12, 2, workload=inputs.WL_PLAIN, start=300)
    T = _dev(batch)
    g = torch.ones((3, 10), device=DEV)
    fwd = qp_forward(*T)
    _, bst = _bwd(fwd, g)
    assert (bst == STATUS_CONVERGED).all()
    # a workspace no forward pass wrote
    fresh = torch.zeros_like(fwd.workspace)
    grads, bst = _bwd(fwd.__class__(**{**fwd.__dict__, "workspace": fresh}), g)
    assert (bst == STATUS_NO_FORWARD).all() and all(torch.isnan(t).all() for t in grads)
    # other Q/G/A buffers than the forward pass's (same values)
    other = fwd.__class__(**{**fwd.__dict__, "Q": fwd.Q.clone(), "G": fwd.G.clone()})
    grads, bst = _bwd(other, g)
    assert (bst == STATUS_NO_FORWARD).all() and torch.isnan(grads[1]).all()
    # a forward on the other kernel path (forced global path) in the same workspace buffer
    opts = default_options(torch.float32)
    opts.path = 1
    ws = alloc_workspace(torch.float32, 3, 10, 12, 2, DEV, opts)
    qp_forward(*T, options=opts, workspace=ws)
    grads, bst = _bwd(fwd.__class__(**{**fwd.__dict__, "workspace": ws}), g)
    assert (bst == STATUS_NO_FORWARD).all()
    # the same workspace with the options it was written with is accepted
    grads, bst = _bwd(fwd.__class__(**{**fwd.__dict__, "workspace": ws, "options": opts}), g)
    assert (bst == STATUS_CONVERGED).all() and torch.isfinite(grads[0]).all()


def test_backward_rejects_a_forward_of_other_sizes():
    small = inputs.random_batch(2, 8, 6, 0, workload=inputs.WL_PLAIN, start=310)
    big = inputs.random_batch(2, 8, 9, 1, workload=inputs.WL_PLAIN, start=320)
    Tb = _dev(big)
    fb = qp_forward(*Tb)
    ws = alloc_workspace(torch.float32, 2, 8, 9, 1, DEV)
    Ts = _dev(small)
    qp_forward(*Ts, workspace=ws)                 # smaller instances written into ws
    grads, bst = _bwd(fb.__class__(**{**fb.__dict__, "workspace": ws}), torch.ones((2, 8), device=DEV))
    assert (bst == STATUS_NO_FORWARD).all()


def test_tensor_core_setup_statuses():
    """At a size whose setup sweep takes the tensor cores: a NaN in Q is caught by the
    superblock's pivot test (NOT_PD or NUMERICAL, NaN outputs, no hang), a NaN in q by the
    residual (NUMERICAL), max_iter = 2 returns a finite iterate, and the other instances of
    the batch converge."""
    from paper_1703_00443_gb300 import STATUS_NOT_PD
    from paper_1703_00443_gb300.qp import uses_tensor_cores
    n, p, m = 140, 200, 30
    assert uses_tensor_cores(torch.float32, n, p, m)
    batch = inputs.random_batch(3, n, p, m, workload=inputs.WL_SWEEP, start=90)
    batch.Q[0, 5, 7] = batch.Q[0, 7, 5] = np.nan
    batch.q[1, 3] = np.nan
    fwd = qp_forward(*_dev(batch))
    grads, bst = _bwd(fwd, torch.ones((3, n), device=DEV))
    st = fwd.status.cpu().numpy()
    assert st[0] in (STATUS_NOT_PD, STATUS_NUMERICAL) and st[1] == STATUS_NUMERICAL, st
    assert st[2] == STATUS_CONVERGED, st
    assert torch.isnan(fwd.z[0]).all() and torch.isnan(fwd.z[1]).all()
    assert torch.isfinite(fwd.z[2]).all() and all(torch.isfinite(t[2]).all() for t in grads)
    opts = default_options(torch.float32)
    opts.max_iter = 2
    batch2 = inputs.random_batch(2, n, p, m, workload=inputs.WL_SWEEP, start=95)
    fwd2 = qp_forward(*_dev(batch2), options=opts)
    grads2, bst2 = _bwd(fwd2, torch.ones((2, n), device=DEV))
    assert (fwd2.status.cpu().numpy() == STATUS_MAX_ITER).all()
    assert torch.isfinite(fwd2.z).all() and all(torch.isfinite(t).all() for t in grads2)
