"""Pins for the FP64 oracle against results that do not come from the oracle itself.

Each pin is fixed by the paper or by mathematics: closed-form layers of the appendix
(ReLU Eq. 21, sum-of-max Eq. 19, three-term max Eq. 24, simplex projection Eq. 25), the
null-space solution of an equality-only QP, brute-force active-set enumeration, the
reduced active-set system from the proof of Theorem 1, the forward-mode Jacobian of the
differentiated KKT system Eq. 6, central finite differences, and the agreement of the two
adjoint derivations (Eq. 7 and Eq. 11).
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_1703_00443_gb300 import inputs


def _rng(k):
    return np.random.default_rng(1000 + k)


def _tiny_qp(r, n, p, m, box=False):
    L = r.standard_normal((n, n))
    Q = L @ L.T + 0.5 * np.eye(n)
    q = r.standard_normal(n)
    if box:
        G = np.vstack([np.eye(n), -np.eye(n)])
        h = np.concatenate([r.uniform(0.1, 1.0, n), r.uniform(0.1, 1.0, n)])
        z0 = r.uniform(-0.05, 0.05, n)   # strictly inside the box
    else:
        G = r.standard_normal((p, n))
        z0 = r.standard_normal(n)
        h = G @ z0 + r.uniform(0.1, 1.0, p)
    A = r.standard_normal((m, n))
    b = A @ z0
    return Q, q, G, h, A, b


# ---------------------------------------------------------------- closed forms / exact solves

def _nullspace_solution(Q, q, A, b):
    """Equality-constrained QP by the null-space method (a different computation from
    the oracle's KKT solve): z = z_p + N w with A z_p = b, AN = 0."""
    zp = np.linalg.lstsq(A, b, rcond=None)[0] if A.shape[0] else np.zeros(Q.shape[0])
    N = sla.null_space(A) if A.shape[0] else np.eye(Q.shape[0])
    w = np.linalg.solve(N.T @ Q @ N, -N.T @ (Q @ zp + q))
    return zp + N @ w


@pytest.mark.parametrize("n,m", [(5, 0), (8, 3), (20, 7)])
def test_equality_only_matches_nullspace(n, m):
    r = _rng(n + m)
    Q, q, _, _, A, b = _tiny_qp(r, n, 0, m)
    G, h = np.zeros((0, n)), np.zeros(0)
    sol = oracle.solve(Q, q, G, h, A, b)
    np.testing.assert_allclose(sol["z"], _nullspace_solution(Q, q, A, b), rtol=0, atol=1e-10)
    if m:
        # stationarity fixes ν uniquely (A full row rank)
        nu = np.linalg.lstsq(A.T, -(Q @ sol["z"] + q), rcond=None)[0]
        np.testing.assert_allclose(sol["nu"], nu, atol=1e-9)


def test_ipm_with_slack_inequalities_reduces_to_equality_qp():
    """Inequalities that stay far from active leave the equality-only solution unchanged
    (λ* → 0), so the interior point path must land on the null-space solution."""
    r = _rng(7)
    n, p, m = 12, 9, 4
    Q, q, _, _, A, b = _tiny_qp(r, n, p, m)
    zeq = _nullspace_solution(Q, q, A, b)
    G = r.standard_normal((p, n))
    h = G @ zeq + r.uniform(5.0, 10.0, p)
    sol = oracle.solve(Q, q, G, h, A, b)
    np.testing.assert_allclose(sol["z"], zeq, atol=1e-10)
    assert np.max(sol["lam"]) < 1e-11


def _active_set_solve(Q, q, G, h, A, b):
    """Brute force over all active sets S: solve the KKT system with G_S z = h_S and keep
    the point that is primal feasible with λ_S ≥ 0 (unique for Q ≻ 0, nondegenerate)."""
    n, p, m = Q.shape[0], G.shape[0], A.shape[0]
    found = []
    for k in range(0, min(p, n - m) + 1):
        for S in itertools.combinations(range(p), k):
            S = list(S)
            GS = G[S]
            N = n + k + m
            K = np.zeros((N, N))
            K[:n, :n] = Q
            K[:n, n:n + k] = GS.T
            K[:n, n + k:] = A.T
            K[n:n + k, :n] = GS
            K[n + k:, :n] = A
            try:
                sol = np.linalg.solve(K, np.concatenate([-q, h[S], b]))
            except np.linalg.LinAlgError:
                continue
            z, lS, nu = sol[:n], sol[n:n + k], sol[n + k:]
            if np.all(G @ z <= h + 1e-10) and np.all(lS >= -1e-10):
                lam = np.zeros(p)
                lam[S] = lS
                found.append((z, lam, nu, S))
    assert found, "no KKT point found by enumeration"
    z0 = found[0][0]
    for f in found[1:]:
        assert np.allclose(f[0], z0, atol=1e-8)
    return found[0]


@pytest.mark.parametrize("k", range(8))
def test_bruteforce_active_set(k):
    r = _rng(100 + k)
    n = 2 + k % 4
    box = (k % 3 == 0)
    p = 2 * n if box else 3 + k
    m = (k % 2) if n > 2 else 0
    Q, q, G, h, A, b = _tiny_qp(r, n, p, m, box=box)
    q = q * 3.0  # push the unconstrained minimiser out so several constraints bind
    z, lam, nu, S = _active_set_solve(Q, q, G, h, A, b)
    sol = oracle.solve(Q, q, G, h, A, b)
    np.testing.assert_allclose(sol["z"], z, atol=1e-9)
    np.testing.assert_allclose(sol["lam"], lam, atol=1e-9)
    if m:
        np.testing.assert_allclose(sol["nu"], nu, atol=1e-9)

    # Limit gradient from the reduced active-set system of the proof of Theorem 1:
    # [Q G_Sᵀ Aᵀ; G_S 0 0; A 0 0][d_z; d̃_S; d_ν] = [−∂ℓ/∂z; 0; 0].
    g = r.standard_normal(n)
    kS = len(S)
    N = n + kS + m
    K = np.zeros((N, N))
    K[:n, :n] = Q
    K[:n, n:n + kS] = G[S].T
    K[:n, n + kS:] = A.T
    K[n:n + kS, :n] = G[S]
    K[n + kS:, :n] = A
    d = np.linalg.solve(K, np.concatenate([-g, np.zeros(kS + m)]))
    dz = d[:n]
    dlt = np.zeros(p)
    dlt[S] = d[n:n + kS]
    gr = oracle.backward(Q, G, h, A, sol, g)
    np.testing.assert_allclose(gr["dq"], dz, atol=1e-8)
    np.testing.assert_allclose(gr["dh"], -dlt, atol=1e-8)
    np.testing.assert_allclose(gr["dG"], np.outer(dlt, z) + np.outer(lam, dz), atol=1e-8)


def test_relu_layer_closed_form():
    """Eq. 21: min ‖z − y‖² s.t. z ≥ 0 is max(y, 0); ∂z/∂y = diag(1[y > 0])."""
    r = _rng(3)
    n = 16
    y = r.standard_normal(n)
    y[np.abs(y) < 0.05] += 0.2  # stay away from the degenerate kink
    Q, q = 2 * np.eye(n), -2 * y
    G, h = -np.eye(n), np.zeros(n)
    A, b = np.zeros((0, n)), np.zeros(0)
    sol = oracle.solve(Q, q, G, h, A, b)
    np.testing.assert_allclose(sol["z"], np.maximum(y, 0), atol=1e-10)
    g = r.standard_normal(n)
    gr = oracle.backward(Q, G, h, A, sol, g)
    # q = −2y, so ∂ℓ/∂q = −½ ∂ℓ/∂y = −½ 1[y>0] g
    np.testing.assert_allclose(gr["dq"], -0.5 * (y > 0) * g, atol=1e-9)


def test_sum_of_max_closed_form():
    """Eq. 19: min ‖t‖² + (z − wᵀt)² s.t. a_i x + b_i ≤ t_i gives t_i = max(a_i x + b_i, 0)
    and z = Σ w_i max(a_i x + b_i, 0)."""
    r = _rng(4)
    k = 7
    w = r.choice([-1.0, 1.0], k)
    a, bb = r.standard_normal(k), r.standard_normal(k)
    for x in (-1.3, 0.4, 2.2):
        u = a * x + bb
        # variables (z, t_1..t_k); objective ½ vᵀQv with Q = 2·[[1, −wᵀ], [−w, I + wwᵀ]]
        Q = np.zeros((k + 1, k + 1))
        Q[0, 0] = 2.0
        Q[0, 1:] = Q[1:, 0] = -2.0 * w
        Q[1:, 1:] = 2.0 * (np.eye(k) + np.outer(w, w))
        q = np.zeros(k + 1)
        G = np.zeros((k, k + 1))
        G[:, 1:] = -np.eye(k)
        h = -u
        sol = oracle.solve(Q, q, G, h, np.zeros((0, k + 1)), np.zeros(0))
        t = np.maximum(u, 0)
        np.testing.assert_allclose(sol["z"][1:], t, atol=1e-9)
        np.testing.assert_allclose(sol["z"][0], w @ t, atol=1e-9)


def test_three_term_max_closed_form():
    """Eq. 24: min z² s.t. a_iᵀx ≤ z (i = 1..3) has z* = max(0, max_i a_iᵀx)."""
    r = _rng(5)
    for trial in range(6):
        a = r.standard_normal((3, 2))
        x = r.standard_normal(2)
        v = a @ x
        Q, q = np.array([[2.0]]), np.zeros(1)
        G, h = -np.ones((3, 1)), -v
        sol = oracle.solve(Q, q, G, h, np.zeros((0, 1)), np.zeros(0))
        assert abs(sol["z"][0] - max(0.0, v.max())) < 1e-9


def _simplex_projection(x):
    """Sort-based Euclidean projection onto the probability simplex (Duchi et al., 2008)."""
    u = np.sort(x)[::-1]
    css = np.cumsum(u) - 1.0
    j = np.arange(1, x.size + 1)
    rho = np.nonzero(u - css / j > 0)[0][-1]
    theta = css[rho] / (rho + 1)
    return np.maximum(x - theta, 0.0)


def test_simplex_projection_closed_form():
    """Eq. 25: min ‖z − x‖² s.t. z ≥ 0, 1ᵀz = 1; Jacobian on the support S is I − 11ᵀ/|S|."""
    r = _rng(6)
    n = 10
    x = r.standard_normal(n)
    zt = _simplex_projection(x)
    Q, q = 2 * np.eye(n), -2 * x
    G, h = -np.eye(n), np.zeros(n)
    A, b = np.ones((1, n)), np.ones(1)
    sol = oracle.solve(Q, q, G, h, A, b)
    np.testing.assert_allclose(sol["z"], zt, atol=1e-10)
    g = r.standard_normal(n)
    S = zt > 1e-12
    J = np.zeros((n, n))
    J[np.ix_(S, S)] = np.eye(S.sum()) - 1.0 / S.sum()
    dldx = J.T @ g
    gr = oracle.backward(Q, G, h, A, sol, g)
    np.testing.assert_allclose(gr["dq"], -0.5 * dldx, atol=1e-9)


# ---------------------------------------------------------------- certificates

@pytest.mark.parametrize("n,p,m", [(10, 20, 0), (30, 30, 15), (1, 3, 0), (6, 2, 5)])
def test_kkt_certificate(n, p, m):
    for i in range(3):
        Q, q, G, h, A, b = inputs.random_qp(n, p, m, index=i, workload=inputs.WL_PLAIN)
        sol = oracle.solve(Q, q, G, h, A, b)
        assert sol["status"] == oracle.STATUS_CONVERGED
        z, lam, nu = sol["z"], sol["lam"], sol["nu"]
        assert np.max(np.abs(Q @ z + q + G.T @ lam + A.T @ nu)) <= 1e-9
        assert np.max(G @ z - h) <= 1e-9
        if m:
            assert np.max(np.abs(A @ z - b)) <= 1e-9
        assert np.min(lam) >= 0
        assert np.max(np.abs(lam * (h - G @ z))) <= 1e-9


# ---------------------------------------------------------------- gradients

def _kkt_diff_forward(Q, G, h, A, sol, dQ, dq, dG, dh, dA, db):
    """Forward-mode differential of the solution from Eq. 6."""
    z, lam, nu = sol["z"], sol["lam"], sol["nu"]
    n, p, m = Q.shape[0], G.shape[0], A.shape[0]
    N = n + p + m
    K = np.zeros((N, N))
    K[:n, :n] = Q
    K[:n, n:n + p] = G.T
    K[:n, n + p:] = A.T
    K[n:n + p, :n] = lam[:, None] * G
    K[n:n + p, n:n + p] = np.diag(G @ z - h)
    K[n + p:, :n] = A
    rhs = -np.concatenate([dQ @ z + dq + dG.T @ lam + dA.T @ nu,
                           lam * (dG @ z) - lam * dh,
                           dA @ z - db])
    return np.linalg.solve(K, rhs)[:n]


@pytest.mark.parametrize("k", range(4))
def test_adjoint_matches_forward_mode_jacobian(k):
    """Substituting each unit dθ in Eq. 6 gives a Jacobian column; its contraction with
    ∂ℓ/∂z must equal the adjoint gradient of Eq. 7-8 (Q perturbed symmetrically)."""
    r = _rng(200 + k)
    n, p, m = 3 + k % 3, 4 + k, k % 2
    Q, q, G, h, A, b = _tiny_qp(r, n, p, m)
    q = 2.5 * q
    sol = oracle.solve(Q, q, G, h, A, b)
    g = r.standard_normal(n)
    gr = oracle.backward(Q, G, h, A, sol, g)
    Z = dict(dQ=np.zeros((n, n)), dq=np.zeros(n), dG=np.zeros((p, n)), dh=np.zeros(p),
             dA=np.zeros((m, n)), db=np.zeros(m))
    for name in Z:
        shape = Z[name].shape
        for idx in np.ndindex(*shape):
            d = {kk: v.copy() for kk, v in Z.items()}
            d[name][idx] = 1.0
            if name == "dQ" and idx[0] != idx[1]:
                d[name][idx[::-1]] = 1.0
            dz = _kkt_diff_forward(Q, G, h, A, sol, **d)
            fwd = g @ dz
            adj = gr[name][idx]
            if name == "dQ" and idx[0] != idx[1]:
                adj = gr[name][idx] + gr[name][idx[::-1]]
            assert abs(fwd - adj) <= 1e-8 * (1 + abs(fwd)), (name, idx, fwd, adj)


def test_central_finite_differences():
    r = _rng(300)
    n, p, m = 5, 7, 2
    Q, q, G, h, A, b = _tiny_qp(r, n, p, m)
    q = 2.0 * q
    g = r.standard_normal(n)
    sol = oracle.solve(Q, q, G, h, A, b)
    gr = oracle.backward(Q, G, h, A, sol, g)
    params = dict(Q=Q, q=q, G=G, h=h, A=A, b=b)

    def loss(pp):
        return g @ oracle.solve(pp["Q"], pp["q"], pp["G"], pp["h"], pp["A"], pp["b"])["z"]

    for name, val in params.items():
        for idx in list(np.ndindex(*val.shape))[::3]:
            eps = 1e-6 * max(1.0, abs(val[idx]))
            plus = {kk: v.copy() for kk, v in params.items()}
            minus = {kk: v.copy() for kk, v in params.items()}
            plus[name][idx] += eps
            minus[name][idx] -= eps
            sym = name == "Q" and idx[0] != idx[1]
            if sym:
                plus[name][idx[::-1]] += eps
                minus[name][idx[::-1]] -= eps
            fd = (loss(plus) - loss(minus)) / (2 * eps)
            adj = gr["d" + name][idx]
            if sym:
                adj = adj + gr["d" + name][idx[::-1]]
            assert abs(fd - adj) <= 1e-6 * (1 + abs(adj)), (name, idx, fd, adj)


def test_central_finite_differences_through_lambda_and_nu():
    """ℓ = g_zᵀz* + g_λᵀλ* + g_νᵀν*: the adjoint with all three right-hand-side blocks matches
    central differences of the oracle's solution (strictly complementary instance)."""
    r = _rng(301)
    n, p, m = 5, 7, 2
    Q, q, G, h, A, b = _tiny_qp(r, n, p, m)
    q = 2.0 * q
    gz, gl, gn = r.standard_normal(n), r.standard_normal(p), r.standard_normal(m)
    sol = oracle.solve(Q, q, G, h, A, b)
    slack = h - G @ sol["z"]
    assert np.min(np.maximum(sol["lam"], slack)) > 1e-3     # strict complementarity
    gr = oracle.backward(Q, G, h, A, sol, gz, gl, gn)
    params = dict(Q=Q, q=q, G=G, h=h, A=A, b=b)

    def loss(pp):
        s2 = oracle.solve(pp["Q"], pp["q"], pp["G"], pp["h"], pp["A"], pp["b"])
        return gz @ s2["z"] + gl @ s2["lam"] + gn @ s2["nu"]

    for name, val in params.items():
        for idx in list(np.ndindex(*val.shape))[::2]:
            eps = 1e-6 * max(1.0, abs(val[idx]))
            plus = {kk: v.copy() for kk, v in params.items()}
            minus = {kk: v.copy() for kk, v in params.items()}
            plus[name][idx] += eps
            minus[name][idx] -= eps
            sym = name == "Q" and idx[0] != idx[1]
            if sym:
                plus[name][idx[::-1]] += eps
                minus[name][idx[::-1]] -= eps
            fd = (loss(plus) - loss(minus)) / (2 * eps)
            adj = gr["d" + name][idx]
            if sym:
                adj = adj + gr["d" + name][idx[::-1]]
            assert abs(fd - adj) <= 1e-6 * (1 + abs(adj)), (name, idx, fd, adj)


@pytest.mark.parametrize("n,p,m", [(10, 20, 3), (6, 11, 2)])
def test_two_adjoint_derivations_agree_with_lambda_and_nu_terms(n, p, m):
    Q, q, G, h, A, b = inputs.random_qp(n, p, m, index=4)
    sol = oracle.solve(Q, q, G, h, A, b)
    r = _rng(302)
    gz, gl, gn = r.standard_normal(n), r.standard_normal(p), r.standard_normal(m)
    g1 = oracle.backward(Q, G, h, A, sol, gz, gl, gn)
    g2 = oracle.backward_sym(Q, G, A, sol, gz, gl, gn)
    for key in ("dQ", "dq", "dG", "dh", "dA", "db"):
        np.testing.assert_allclose(g1[key], g2[key], rtol=1e-7, atol=1e-9, err_msg=key)


@pytest.mark.parametrize("n,p,m", [(10, 20, 0), (20, 20, 10), (4, 9, 1)])
def test_two_adjoint_derivations_agree(n, p, m):
    """Eq. 7 (transposed Eq. 6 matrix) and Eq. 11 (symmetrised K) give the same d_z, d̃_λ,
    d_ν and therefore the same gradients."""
    Q, q, G, h, A, b = inputs.random_qp(n, p, m, index=3)
    sol = oracle.solve(Q, q, G, h, A, b)
    g = inputs.upstream_grad(1, n)[0].astype(np.float64)
    g1 = oracle.backward(Q, G, h, A, sol, g)
    g2 = oracle.backward_sym(Q, G, A, sol, g)
    for key in ("dQ", "dq", "dG", "dh", "dA", "db"):
        np.testing.assert_allclose(g1[key], g2[key], rtol=1e-7, atol=1e-9, err_msg=key)


def test_degenerate_small_sizes():
    # n = 1 with one active and one inactive bound
    Q, q = np.array([[1.0]]), np.array([-3.0])
    G, h = np.array([[1.0], [-1.0]]), np.array([1.0, 5.0])
    sol = oracle.solve(Q, q, G, h, np.zeros((0, 1)), np.zeros(0))
    assert abs(sol["z"][0] - 1.0) < 1e-10
    assert abs(sol["lam"][0] - 2.0) < 1e-9 and sol["lam"][1] < 1e-10
