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


def rel_err_inf(x, ref, floor=None):
    """Per-instance max_i |x_i − ref_i| / max(‖ref‖∞, floor), the ∞-norm form of rel_err."""
    x = np.asarray(x, dtype=np.float64).reshape(len(x), -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(len(ref), -1)
    if x.shape[1] == 0:
        return np.zeros(len(x))
    fl = 1e-12 if floor is None else np.maximum(np.asarray(floor, dtype=np.float64), 1e-12)
    return np.max(np.abs(x - ref), axis=1) / np.maximum(np.max(np.abs(ref), axis=1), fl)


MATRIX_GRADS = ("dQ", "dG", "dA")


def grad_floor(name, dl_dz, z_ref, norm=2):
    """Denominator floor for a gradient's relative error.  A gradient can vanish
    identically at the solution (e.g. ∂z*/∂q = 0 when n constraints are active), where a
    plain relative error is undefined; the floor is 1e-3·‖∂ℓ/∂z*‖, times max(1, ‖z*‖) for
    the outer-product gradients dQ, dG, dA (2-norms, or ∞-norms with norm=inf)."""
    ord_ = None if norm == 2 else np.inf
    g = np.linalg.norm(np.asarray(dl_dz, dtype=np.float64).reshape(len(dl_dz), -1), ord=ord_, axis=1)
    if name in MATRIX_GRADS:
        zn = np.linalg.norm(np.asarray(z_ref, dtype=np.float64).reshape(len(z_ref), -1), ord=ord_,
                            axis=1)
        return 1e-3 * g * np.maximum(1.0, zn)
    return 1e-3 * g


def _oracle_one(args):
    Q, q, G, h, A, b, g = args
    sol = oracle.solve(Q, q, G, h, A, b)
    return sol, oracle.backward(Q, G, h, A, sol, g)


def oracle_many(problems, workers=None):
    """Oracle solution and gradients of each (Q, q, G, h, A, b, dl_dz) tuple (FP64).  Many
    problems go to a pool of worker processes (started with spawn, never forked, so it is
    safe after CUDA was initialised), one BLAS thread each."""
    problems = [tuple(np.asarray(x, dtype=np.float64) for x in pr) for pr in problems]
    if len(problems) < 16:
        return [_oracle_one(pr) for pr in problems]
    import multiprocessing as mp
    import os
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(workers or min(len(problems), os.cpu_count() or 1)) as pool:
            return pool.map(_oracle_one, problems)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def oracle_solve_and_grad(batch, dl_dz, idx=None):
    """Oracle z*, λ*, ν*, gradients for the selected instances (all by default)."""
    idx = list(range(batch.B) if idx is None else idx)
    res = oracle_many([batch.instance(i) + (np.asarray(dl_dz[i], dtype=np.float64),)
                       for i in idx])
    sols = [r[0] for r in res]
    assert all(s["status"] == oracle.STATUS_CONVERGED for s in sols)
    return sols, [r[1] for r in res]


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
