"""Writes closed_forms.json: small QPs whose solution (and, where the paper gives it, the
gradient of a loss through the solution) has a closed form stated in the paper's appendix.
The expected values are those closed forms evaluated in FP64 with NumPy; nothing here calls
the oracle or the CUDA path.  Run from the repository root:

    python tests/golden/make_closed_forms.py
"""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _rng(k):
    return np.random.Generator(np.random.Philox(key=[20170301, k]))


def _case(name, cite, Q, q, G, h, A, b, z, g=None, dq=None):
    c = {"name": name, "cite": cite, "n": int(Q.shape[0]), "nineq": int(G.shape[0]),
         "neq": int(A.shape[0])}
    for k, v in (("Q", Q), ("q", q), ("G", G), ("h", h), ("A", A), ("b", b), ("z", z)):
        c[k] = np.asarray(v, dtype=np.float64).reshape(-1).tolist()
    if g is not None:
        c["dl_dz"] = np.asarray(g, dtype=np.float64).tolist()
        c["dq"] = np.asarray(dq, dtype=np.float64).tolist()
    return c


def relu(r, n):
    # Appendix, Eq. 21: min ‖z − y‖² s.t. z ≥ 0 gives z = max(y, 0), ∂z/∂y = diag(1[y > 0]);
    # with q = −2y, ∂ℓ/∂q = −½ 1[y > 0] ∘ ∂ℓ/∂z.
    y = r.standard_normal(n)
    y[np.abs(y) < 0.1] += 0.3          # strictly complementary (no kink at the solution)
    g = r.standard_normal(n)
    return _case(f"relu_n{n}", "appendix Eq. 21 (Theorem 2 proof)", 2 * np.eye(n), -2 * y,
                 -np.eye(n), np.zeros(n), np.zeros((0, n)), np.zeros(0), np.maximum(y, 0), g,
                 -0.5 * (y > 0) * g)


def sum_of_max(r, k, x):
    # Appendix, Eq. 19: min ‖t‖² + (z − wᵀt)² s.t. a_i x + b_i ≤ t_i gives
    # t_i = max(a_i x + b_i, 0), z = Σ_i w_i t_i.  Variables v = (z, t).
    w = r.choice([-1.0, 1.0], k)
    a, bb = r.standard_normal(k), r.standard_normal(k)
    u = a * x + bb
    u[np.abs(u) < 0.1] += 0.3
    Q = np.zeros((k + 1, k + 1))
    Q[0, 0] = 2.0
    Q[0, 1:] = Q[1:, 0] = -2.0 * w
    Q[1:, 1:] = 2.0 * (np.eye(k) + np.outer(w, w))
    G = np.zeros((k, k + 1))
    G[:, 1:] = -np.eye(k)
    t = np.maximum(u, 0)
    return _case(f"sum_of_max_k{k}_x{x:+.1f}", "appendix Eq. 19 (Theorem 2 proof)", Q,
                 np.zeros(k + 1), G, -u, np.zeros((0, k + 1)), np.zeros(0),
                 np.concatenate([[w @ t], t]))


def three_term_max(r, tag):
    # Appendix, Eq. 24: min z² s.t. a_iᵀx ≤ z (i = 1..3) gives z = max(0, max_i a_iᵀx)
    # (the appendix writes max_i a_iᵀx; the QP's solution clips at 0).
    a = r.standard_normal((3, 2))
    x = r.standard_normal(2)
    v = a @ x
    return _case(f"three_term_max_{tag}", "appendix Eq. 24 (Theorem 3 proof)", np.array([[2.0]]),
                 np.zeros(1), -np.ones((3, 1)), -v, np.zeros((0, 1)), np.zeros(0),
                 np.array([max(0.0, v.max())]))


def simplex(r, n):
    # Appendix, Eq. 25: min ‖z − x‖² s.t. z ≥ 0, 1ᵀz = 1 is the Euclidean projection onto
    # the simplex (sort-based method of Duchi et al. 2008, which the appendix cites); on the
    # support S the Jacobian is I − 11ᵀ/|S|, so ∂ℓ/∂q = −½ Jᵀ ∂ℓ/∂z with q = −2x.
    x = r.standard_normal(n)
    u = np.sort(x)[::-1]
    css = np.cumsum(u) - 1.0
    j = np.arange(1, n + 1)
    rho = np.nonzero(u - css / j > 0)[0][-1]
    theta = css[rho] / (rho + 1)
    z = np.maximum(x - theta, 0.0)
    S = z > 1e-12
    assert np.min(np.abs(x - theta)) > 1e-3          # strictly complementary
    J = np.zeros((n, n))
    J[np.ix_(S, S)] = np.eye(S.sum()) - 1.0 / S.sum()
    g = r.standard_normal(n)
    return _case(f"simplex_n{n}", "appendix Eq. 25", 2 * np.eye(n), -2 * x, -np.eye(n),
                 np.zeros(n), np.ones((1, n)), np.ones(1), z, g, -0.5 * (J.T @ g))


def main():
    cases = [relu(_rng(1), 16), relu(_rng(2), 40)]
    cases += [sum_of_max(_rng(3), 7, x) for x in (-1.3, 0.4, 2.2)]
    cases += [three_term_max(_rng(4 + k), k) for k in range(3)]
    cases += [simplex(_rng(10), 10), simplex(_rng(11), 24)]
    with open(os.path.join(HERE, "closed_forms.json"), "w") as f:
        json.dump({"about": "closed-form QP layers of the paper's appendix; expected values "
                            "are the closed forms (see make_closed_forms.py)",
                   "cases": cases}, f, indent=1)


if __name__ == "__main__":
    main()
