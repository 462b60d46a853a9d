"""Shared test helpers: run the CUDA path and the oracle on the same seeded inputs."""
import numpy as np

import oracle


def rel_err(x, ref, floor=None):
    """Per-instance ‖x − ref‖₂ / max(‖ref‖₂, floor) (rows = instances); floor defaults to
    1e-12 and may be a per-instance array."""
    x = np.asarray(x, dtype=np.float64).reshape(len(x), -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(len(ref), -1)
    if x.shape[1] == 0:
        return np.zeros(len(x))
    fl = 1e-12 if floor is None else np.maximum(np.asarray(floor, dtype=np.float64), 1e-12)
    return np.linalg.norm(x - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), fl)


MATRIX_GRADS = ("dQ", "dG", "dA")


def grad_floor(name, dl_dz, z_ref):
    """Denominator floor for a gradient's relative error.  A gradient can vanish
    identically at the solution (e.g. ∂z*/∂q = 0 when n constraints are active), where a
    plain relative error is undefined; the floor is 1e-3·‖∂ℓ/∂z*‖₂, times max(1, ‖z*‖₂) for
    the outer-product gradients dQ, dG, dA."""
    g = np.linalg.norm(np.asarray(dl_dz, dtype=np.float64).reshape(len(dl_dz), -1), axis=1)
    if name in MATRIX_GRADS:
        zn = np.linalg.norm(np.asarray(z_ref, dtype=np.float64).reshape(len(z_ref), -1), axis=1)
        return 1e-3 * g * np.maximum(1.0, zn)
    return 1e-3 * g


def oracle_solve_and_grad(batch, dl_dz, idx=None):
    """Oracle z*, λ*, ν*, gradients for the selected instances (all by default)."""
    idx = range(batch.B) if idx is None else idx
    sols, grads = [], []
    for i in idx:
        Q, q, G, h, A, b = batch.instance(i)
        sol = oracle.solve(Q, q, G, h, A, b)
        assert sol["status"] == oracle.STATUS_CONVERGED
        sols.append(sol)
        grads.append(oracle.backward(Q, G, h, A, sol, np.asarray(dl_dz[i], dtype=np.float64)))
    return sols, grads


def kkt_residuals_fp64(batch, z, lam, nu):
    """FP64 KKT residuals of returned (z, λ, ν) for every instance, scaled like the solver's
    stopping test: stationarity, primal feasibility, complementarity, dual sign."""
    out = []
    for i in range(batch.B):
        Q, q, G, h, A, b = batch.instance(i)
        zi, li, ni = (np.asarray(v[i], dtype=np.float64) for v in (z, lam, nu))
        rz = np.max(np.abs(Q @ zi + q + G.T @ li + A.T @ ni)) / (1 + np.max(np.abs(q)))
        slack = h - G @ zi if G.shape[0] else np.zeros(0)
        rp = max(np.max(-slack, initial=0.0), np.max(np.abs(A @ zi - b), initial=0.0)) / (
            1 + np.max(np.abs(h), initial=0.0) + np.max(np.abs(b), initial=0.0))
        comp = np.max(np.abs(li * slack), initial=0.0)
        dsign = np.max(-li, initial=0.0)
        out.append((rz, rp, comp, dsign))
    return np.array(out)
