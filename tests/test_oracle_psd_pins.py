"""Pins for the oracle on positive semidefinite Q (§3, Eq. 2 allows Q ⪰ 0): linear programs
(Q = 0) and QPs whose Q is rank deficient, including the TV-denoising QP of §4.2.  None of the
reference values comes from the oracle:

* an LP's optimum by enumerating its vertices (the optimum of a bounded LP with a unique
  solution is a vertex), and at that vertex the closed-form gradient of ℓ = gᵀz*: with the
  active rows C = [G_S; A] (square, invertible at a nondegenerate vertex) z* = C⁻¹[h_S; b],
  so ∂ℓ/∂[h_S; b] = C⁻ᵀg, ∂ℓ/∂h_i = 0 off S, ∂ℓ/∂q = 0, ∂ℓ/∂G_S = −(C⁻ᵀg)_S z*ᵀ and
  ∂ℓ/∂A = −(C⁻ᵀg)_A z*ᵀ;
* brute-force active-set enumeration for rank-deficient Q (the KKT point of each candidate
  active set, kept if primal feasible with λ ≥ 0);
* the TV-denoising QP (min ½‖y − z‖² + w Σ|z_{i+1} − z_i|, slack form) against the same
  enumeration.
"""
import itertools

import numpy as np
import pytest

import oracle
from tests.test_oracle_pins import _active_set_solve


def _rng(k):
    return np.random.default_rng(5000 + k)


def _box_lp(r, n, p_extra, m):
    """LP with a box [−1, 1]ⁿ and p_extra random rows through an interior point."""
    G = np.vstack([np.eye(n), -np.eye(n), r.standard_normal((p_extra, n))])
    z0 = r.uniform(-0.3, 0.3, n)
    h = np.concatenate([np.ones(2 * n), G[2 * n:] @ z0 + r.uniform(0.2, 1.0, p_extra)])
    A = r.standard_normal((m, n))
    b = A @ z0
    q = r.standard_normal(n)
    return np.zeros((n, n)), q, G, h, A, b


def _lp_vertex(q, G, h, A, b):
    """Optimal vertex of min qᵀz s.t. Gz ≤ h, Az = b by enumeration: every choice of n − m rows
    of G that with A fixes a unique point, kept if feasible; the feasible vertex of least
    objective (unique for generic q).  Returns z*, the active rows S and C = [G_S; A]."""
    n, m = G.shape[1], A.shape[0]
    best = None
    for S in itertools.combinations(range(G.shape[0]), n - m):
        C = np.vstack([G[list(S)], A])
        if abs(np.linalg.det(C)) < 1e-10:
            continue
        z = np.linalg.solve(C, np.concatenate([h[list(S)], b]))
        if np.all(G @ z <= h + 1e-9):
            f = q @ z
            if best is None or f < best[0] - 1e-12:
                best = (f, z, list(S), C)
    assert best is not None
    return best[1], best[2], best[3]


@pytest.mark.parametrize("k", range(6))
def test_lp_optimum_is_the_best_vertex_and_gradients_are_the_vertex_ones(k):
    r = _rng(k)
    n = 2 + k % 3
    m = k % 2
    Q, q, G, h, A, b = _box_lp(r, n, 2 + k % 2, m)
    z, S, C = _lp_vertex(q, G, h, A, b)
    sol = oracle.solve(Q, q, G, h, A, b)
    assert sol["status"] == oracle.STATUS_CONVERGED
    np.testing.assert_allclose(sol["z"], z, atol=1e-8)
    g = r.standard_normal(n)
    gr = oracle.backward(Q, G, h, A, sol, g)
    w = np.linalg.solve(C.T, g)            # ∂ℓ/∂[h_S; b]
    dh = np.zeros(G.shape[0])
    dh[S] = w[:len(S)]
    np.testing.assert_allclose(gr["dq"], np.zeros(n), atol=1e-7)
    np.testing.assert_allclose(gr["dh"], dh, atol=1e-7)
    np.testing.assert_allclose(gr["dG"], -np.outer(dh, z), atol=1e-7)
    if m:
        np.testing.assert_allclose(gr["db"], w[len(S):], atol=1e-7)
        np.testing.assert_allclose(gr["dA"], -np.outer(w[len(S):], z), atol=1e-7)


@pytest.mark.parametrize("k", range(6))
def test_rank_deficient_q_matches_active_set_enumeration(k):
    r = _rng(100 + k)
    n = 3 + k % 2
    rank = 1 + k % 2
    L = r.standard_normal((n, rank))
    Q = L @ L.T
    q = 3.0 * r.standard_normal(n)
    G = np.vstack([np.eye(n), -np.eye(n)])
    h = r.uniform(0.3, 1.0, 2 * n)
    m = k % 2
    A = r.standard_normal((m, n))
    b = A @ r.uniform(-0.1, 0.1, n)
    z, lam, nu, S = _active_set_solve(Q, q, G, h, A, b)
    sol = oracle.solve(Q, q, G, h, A, b)
    assert sol["status"] == oracle.STATUS_CONVERGED
    np.testing.assert_allclose(sol["z"], z, atol=1e-8)
    np.testing.assert_allclose(sol["lam"], lam, atol=1e-7)


def tv_qp(y, w):
    """TV denoising (§4.2), min ½‖y − z‖² + w Σ_i |z_{i+1} − z_i|, as a QP in (z, t):
    Q = diag(I, 0), q = (−y, w·1), rows Dz − t ≤ 0 and −Dz − t ≤ 0 (D the first difference)."""
    n = len(y)
    D = np.diff(np.eye(n), axis=0)
    k = n - 1
    Q = np.zeros((n + k, n + k))
    Q[:n, :n] = np.eye(n)
    q = np.concatenate([-y, w * np.ones(k)])
    G = np.block([[D, -np.eye(k)], [-D, -np.eye(k)]])
    h = np.zeros(2 * k)
    return Q, q, G, h, np.zeros((0, n + k)), np.zeros(0)


@pytest.mark.parametrize("seed", range(4))
def test_tv_denoising_qp_matches_active_set_enumeration(seed):
    r = _rng(200 + seed)
    y = r.standard_normal(4)
    Q, q, G, h, A, b = tv_qp(y, 0.3)
    z, lam, nu, S = _active_set_solve(Q, q, G, h, A, b)
    sol = oracle.solve(Q, q, G, h, A, b)
    assert sol["status"] == oracle.STATUS_CONVERGED
    np.testing.assert_allclose(sol["z"], z, atol=1e-8)
    # the denoised signal moves toward the mean and its total variation shrinks
    zs = sol["z"][:4]
    assert np.abs(np.diff(zs)).sum() <= np.abs(np.diff(y)).sum() + 1e-9
