"""FP64 CPU oracle for the batched differentiable QP of OptNet (Amos & Kolter, 2017).

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call or execute this
module: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it. It shares no code with the CUDA path.

What it computes, each function citing the passage it follows:

* ``solve``     -- the primal-dual interior point method of §3.1 (slack form, affine
                   predictor Eq. 9, centering-plus-corrector Eq. 10, combined step), run in
                   FP64 on the *full, unreduced* KKT matrix K of Eq. 9 with a dense LU
                   solve (no block elimination, no FP32), to a tight tolerance.
* ``backward``  -- the adjoint system Eq. 7 and the parameter gradients Eq. 8.
* ``backward_sym`` -- the same quantities through the symmetrised system Eq. 11 of §3.1.1
                   (a second derivation; the two must agree).

Readings where the paper is silent (the same readings the CUDA path takes):

* σ (only "as in CVXGEN"): Mehrotra's σ = (μ_aff/μ)³.
* step size ("an appropriate step size"): one fraction-to-boundary step for all variables,
  α = min(1, 0.99·sup{α : s + αΔs ≥ 0, λ + αΔλ ≥ 0}); α_aff = min(1, sup{…}) without 0.99.
* initial point: the CVXOPT start -- solve the KKT system with D(s/λ) = I, i.e.
  [Q Gᵀ Aᵀ; G −I 0; A 0 0][z; λ̂; ν] = [−q; h; b]; then s = −λ̂ and λ = λ̂, each shifted
  by (1 + max(−v)) when max(−v) ≥ −1e-8·max(‖v‖₂, 1).
* stopping: ‖r_z‖∞ ≤ tol·(1+‖q‖∞), ‖r_λ‖∞ ≤ tol·(1+‖h‖∞), ‖r_ν‖∞ ≤ tol·(1+‖b‖∞) and
  μ ≤ mu_tol; at most ``max_iter`` Newton steps.
* nineq = 0: no interior point iterations; the equality-constrained KKT system is solved
  directly.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

STATUS_CONVERGED = 0
STATUS_MAX_ITER = 1


def residuals(Q, q, G, h, A, b, z, s, lam, nu):
    """KKT residuals of the slack form, the right-hand side of Eq. 9 (negated):
    r_z = Qz + q + Gᵀλ + Aᵀν, r_λ = Gz + s − h, r_ν = Az − b; μ = sᵀλ/nineq (§3.1)."""
    rz = Q @ z + q + G.T @ lam + A.T @ nu
    rl = G @ z + s - h
    rn = A @ z - b
    mu = float(s @ lam) / max(G.shape[0], 1)
    return rz, rl, rn, mu


def kkt_matrix(Q, G, A, s, lam):
    """The matrix K of Eq. 9, unknowns ordered (Δz, Δs, Δλ, Δν)."""
    n, p, m = Q.shape[0], G.shape[0], A.shape[0]
    N = n + 2 * p + m
    K = np.zeros((N, N))
    iz, is_, il, iv = slice(0, n), slice(n, n + p), slice(n + p, n + 2 * p), slice(n + 2 * p, N)
    K[iz, iz] = Q
    K[iz, il] = G.T
    K[iz, iv] = A.T
    K[is_, is_] = np.diag(lam)
    K[is_, il] = np.diag(s)
    K[il, iz] = G
    K[il, is_] = np.eye(p)
    K[iv, iz] = A
    return K


def _split(x, n, p, m):
    return x[:n], x[n:n + p], x[n + p:n + 2 * p], x[n + 2 * p:n + 2 * p + m]


def max_step(v, dv):
    """sup{α ≥ 0 : v + α·dv ≥ 0} (inf if no component decreases)."""
    neg = dv < 0
    if not np.any(neg):
        return np.inf
    return float(np.min(-v[neg] / dv[neg]))


def _shift_positive(v):
    """CVXOPT's shift of a starting vector into the interior of the orthant."""
    t = float(np.max(-v))
    if t >= -1e-8 * max(float(np.linalg.norm(v)), 1.0):
        v = v + (1.0 + t)
    return v


def initial_point(Q, q, G, h, A, b):
    """Starting point (reading of §3.1, which does not state one): the KKT solve with
    D(s/λ) = I, then both s and λ shifted into the positive orthant."""
    n, p, m = Q.shape[0], G.shape[0], A.shape[0]
    K = np.zeros((n + p + m, n + p + m))
    K[:n, :n] = Q
    K[:n, n:n + p] = G.T
    K[:n, n + p:] = A.T
    K[n:n + p, :n] = G
    K[n:n + p, n:n + p] = -np.eye(p)
    K[n + p:, :n] = A
    sol = np.linalg.solve(K, np.concatenate([-q, h, b]))
    z, lhat, nu = sol[:n], sol[n:n + p], sol[n + p:]
    return z, _shift_positive(-lhat), _shift_positive(lhat.copy()), nu


def solve(Q, q, G, h, A, b, *, tol=1e-12, mu_tol=1e-13, max_iter=100):
    """Mehrotra predictor-corrector PDIPM of §3.1 in FP64.

    Returns a dict with z, s, lam, nu, iters (Newton steps taken) and status.
    """
    Q, q, G, h, A, b = (np.asarray(x, dtype=np.float64) for x in (Q, q, G, h, A, b))
    n, p, m = Q.shape[0], G.shape[0], A.shape[0]
    if p == 0:
        K = np.zeros((n + m, n + m))
        K[:n, :n] = Q
        K[:n, n:] = A.T
        K[n:, :n] = A
        sol = np.linalg.solve(K, np.concatenate([-q, b]))
        return dict(z=sol[:n], s=np.zeros(0), lam=np.zeros(0), nu=sol[n:], iters=0,
                    status=STATUS_CONVERGED)

    z, s, lam, nu = initial_point(Q, q, G, h, A, b)
    sq, sh, sb = (1.0 + (np.max(np.abs(x)) if x.size else 0.0) for x in (q, h, b))
    status = STATUS_MAX_ITER
    it = 0
    for it in range(max_iter + 1):
        rz, rl, rn, mu = residuals(Q, q, G, h, A, b, z, s, lam, nu)
        if (np.max(np.abs(rz)) <= tol * sq and np.max(np.abs(rl)) <= tol * sh
                and (m == 0 or np.max(np.abs(rn)) <= tol * sb) and mu <= mu_tol):
            status = STATUS_CONVERGED
            break
        if it == max_iter:
            break
        lu = sla.lu_factor(kkt_matrix(Q, G, A, s, lam))
        # Affine-scaling (predictor) direction, Eq. 9.
        rhs = -np.concatenate([rz, s * lam, rl, rn])
        dz_a, ds_a, dl_a, dn_a = _split(sla.lu_solve(lu, rhs), n, p, m)
        a_aff = min(1.0, max_step(s, ds_a), max_step(lam, dl_a))
        mu_aff = float((s + a_aff * ds_a) @ (lam + a_aff * dl_a)) / p
        sigma = (mu_aff / mu) ** 3
        # Centering-plus-corrector direction, Eq. 10, with the same K.
        rhs_cc = np.concatenate([np.zeros(n), sigma * mu - ds_a * dl_a, np.zeros(p), np.zeros(m)])
        dz_c, ds_c, dl_c, dn_c = _split(sla.lu_solve(lu, rhs_cc), n, p, m)
        dz, ds, dl, dn = dz_a + dz_c, ds_a + ds_c, dl_a + dl_c, dn_a + dn_c
        alpha = min(1.0, 0.99 * min(max_step(s, ds), max_step(lam, dl)))
        z = z + alpha * dz
        s = s + alpha * ds
        lam = lam + alpha * dl
        nu = nu + alpha * dn
    return dict(z=z, s=s, lam=lam, nu=nu, iters=it, status=status)


def _grads(z, lam, nu, dz, dlt, dnu):
    """Parameter gradients of Eq. 8, written with d̃_λ = D(λ*)d_λ."""
    return dict(
        dQ=0.5 * (np.outer(dz, z) + np.outer(z, dz)),
        dq=dz.copy(),
        dG=np.outer(dlt, z) + np.outer(lam, dz),
        dh=-dlt,
        dA=np.outer(dnu, z) + np.outer(nu, dz),
        db=-dnu,
    )


def backward(Q, G, h, A, sol, dl_dz, dl_dlam=None, dl_dnu=None):
    """Adjoint solve of Eq. 7 at the solution and gradients of Eq. 8.

    [d_z; d_λ; d_ν] = −[[Q, GᵀD(λ*), Aᵀ], [G, D(Gz*−h), 0], [A, 0, 0]]⁻¹
                       [(∂ℓ/∂z*)ᵀ; (∂ℓ/∂λ*)ᵀ; (∂ℓ/∂ν*)ᵀ].
    Eq. 7 as printed has zeros in the last two blocks (the paper does not differentiate
    through λ*, ν*); a loss that depends on them puts its derivatives there (chain rule
    through the same implicit differentiation of Eq. 6), and Eq. 8 is unchanged.
    Returns the six gradients plus d_z, d_λ, d̃_λ = D(λ*)d_λ and d_ν.
    """
    Q, G, h, A = (np.asarray(x, dtype=np.float64) for x in (Q, G, h, A))
    z, lam, nu = sol["z"], sol["lam"], sol["nu"]
    n, p, m = Q.shape[0], G.shape[0], A.shape[0]
    N = n + p + m
    K = np.zeros((N, N))
    K[:n, :n] = Q
    K[:n, n:n + p] = G.T * lam[None, :]
    K[:n, n + p:] = A.T
    K[n:n + p, :n] = G
    K[n:n + p, n:n + p] = np.diag(G @ z - h)
    K[n + p:, :n] = A
    gl = np.zeros(p) if dl_dlam is None else np.asarray(dl_dlam, dtype=np.float64)
    gn = np.zeros(m) if dl_dnu is None else np.asarray(dl_dnu, dtype=np.float64)
    rhs = np.concatenate([np.asarray(dl_dz, dtype=np.float64), gl, gn])
    d = -np.linalg.solve(K, rhs)
    dz, dl, dnu = d[:n], d[n:n + p], d[n + p:]
    dlt = lam * dl
    out = _grads(z, lam, nu, dz, dlt, dnu)
    out.update(d_z=dz, d_lam=dl, d_lam_tilde=dlt, d_nu=dnu)
    return out


def backward_sym(Q, G, A, sol, dl_dz, dl_dlam=None, dl_dnu=None):
    """The same adjoint through the symmetrised KKT matrix of §3.1.1, Eq. 11:
    K_sym [d_z; d_s; d̃_λ; d_ν] = [−∂ℓ/∂z*; 0; −∂ℓ/∂λ*; −∂ℓ/∂ν*], K_sym = K of Eq. 9 with
    its second block row scaled by D(1/s).  (Eliminating d_s from rows 2 and 3 gives
    G d_z − D(s/λ) d̃_λ = −∂ℓ/∂λ*, which is the λ row of Eq. 7 written in d̃_λ = D(λ*) d_λ.)"""
    Q, G, A = (np.asarray(x, dtype=np.float64) for x in (Q, G, A))
    z, s, lam, nu = sol["z"], sol["s"], sol["lam"], sol["nu"]
    n, p, m = Q.shape[0], G.shape[0], A.shape[0]
    K = kkt_matrix(Q, G, A, s, lam)
    K[n:n + p, :] /= s[:, None]
    gl = np.zeros(p) if dl_dlam is None else np.asarray(dl_dlam, dtype=np.float64)
    gn = np.zeros(m) if dl_dnu is None else np.asarray(dl_dnu, dtype=np.float64)
    rhs = np.concatenate([-np.asarray(dl_dz, dtype=np.float64), np.zeros(p), -gl, -gn])
    dz, ds, dlt, dnu = _split(np.linalg.solve(K, rhs), n, p, m)
    out = _grads(z, lam, nu, dz, dlt, dnu)
    out.update(d_z=dz, d_s=ds, d_lam_tilde=dlt, d_nu=dnu)
    return out


def solve_batch(batch, **kw):
    """Solve every instance of an ``inputs.QPBatch``-like object (FP64)."""
    return [solve(*batch.instance(i), **kw) for i in range(batch.B)]


def backward_batch(batch, sols, dl_dz):
    outs = []
    for i in range(batch.B):
        Q, q, G, h, A, b = batch.instance(i)
        outs.append(backward(Q, G, h, A, sols[i], np.asarray(dl_dz[i], dtype=np.float64)))
    return outs
