"""Seeded synthetic QP generators shared by the tests, the bench and the oracle's callers.

This module only *builds problem data*; it contains none of the solver's arithmetic, so
both the CUDA path and the FP64 oracle can be fed from it without sharing method code.

Every instance is drawn from its own counter-keyed stream
``SeedSequence([seed, workload_id, index])`` so that an instance's data never depends
on how a batch is composed (the same QP alone or in a mix is bit-identical).

Data are drawn in FP64 and then rounded once to the storage dtype; callers hand the
*rounded* values (cast back to FP64) to the oracle, so both sides solve the same problem.

Problem form (Eq. 2, §3): minimise ½zᵀQz + qᵀz subject to Az = b, Gz ≤ h, with
``nineq`` rows in G and ``neq`` rows in A.

The random-QP recipe follows the timing experiment of §4.1 (its footnote: Q = UᵀU + 1e-3·I,
G normal, h = G z0 + s0 with z0 normal and s0 uniform, which makes every instance strictly
feasible), with L ~ N(0,1)/√n in place of the uniform U and with optional equality rows
A ~ N(0,1), b = A z0.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Workload ids used as the second key of every instance stream.
WL_PLAIN = 0        # random dense QP, recipe of the §4.1 timing experiment
WL_SWEEP = 1        # same recipe at the timing-sweep sizes
WL_ONEHOT = 2       # structured one-hot QP (Q = 0.1 I, z >= 0, dense equalities)
WL_UNEVEN = 3       # uneven batch: per-instance sizes drawn too
WL_SERVE = 4        # serving stream
WL_PSD = 5          # positive semidefinite Q (LPs with rank 0)
WL_TV = 6           # total-variation denoising (§4.2) on synthetic signals


@dataclasses.dataclass
class QPBatch:
    """A batch of equally sized QPs, arrays stacked on axis 0 (row-major)."""

    Q: np.ndarray   # [B, n, n]
    q: np.ndarray   # [B, n]
    G: np.ndarray   # [B, nineq, n]
    h: np.ndarray   # [B, nineq]
    A: np.ndarray   # [B, neq, n]
    b: np.ndarray   # [B, neq]

    @property
    def B(self) -> int:
        return self.Q.shape[0]

    @property
    def n(self) -> int:
        return self.Q.shape[1]

    @property
    def nineq(self) -> int:
        return self.G.shape[1]

    @property
    def neq(self) -> int:
        return self.A.shape[1]

    def astype(self, dtype) -> "QPBatch":
        return QPBatch(*(np.ascontiguousarray(x, dtype=dtype) for x in
                         (self.Q, self.q, self.G, self.h, self.A, self.b)))

    def instance(self, i: int):
        """(Q, q, G, h, A, b) of instance i as FP64 arrays."""
        return tuple(np.asarray(x[i], dtype=np.float64) for x in
                     (self.Q, self.q, self.G, self.h, self.A, self.b))


def _rng(seed: int, workload: int, index: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, workload, index])))


def _round(x: np.ndarray, dtype) -> np.ndarray:
    return np.asarray(x, dtype=dtype).astype(np.float64)


def random_qp(n: int, nineq: int, neq: int, *, seed: int = 0, workload: int = WL_PLAIN,
              index: int = 0, dtype=np.float32):
    """One strictly feasible random QP; returns FP64 arrays already rounded to ``dtype``.

    Q = L Lᵀ + 1e-3·I with L ~ N(0,1)/√n; q ~ N(0,1); G ~ N(0,1); z0 ~ N(0,1);
    s0 ~ U(0.5, 1.5); h = G z0 + s0; A ~ N(0,1) (full row rank almost surely); b = A z0.
    Q is symmetrised before rounding so the rounded matrix is exactly symmetric.
    """
    r = _rng(seed, workload, index)
    L = r.standard_normal((n, n)) / math.sqrt(n)
    Q = L @ L.T + 1e-3 * np.eye(n)
    Q = 0.5 * (Q + Q.T)
    q = r.standard_normal(n)
    G = r.standard_normal((nineq, n))
    z0 = r.standard_normal(n)
    s0 = r.uniform(0.5, 1.5, nineq)
    A = r.standard_normal((neq, n))
    Q, q, G, A = (_round(x, dtype) for x in (Q, q, G, A))
    z0 = _round(z0, dtype)
    h = _round(G @ z0 + s0, dtype)
    b = _round(A @ z0, dtype)
    return Q, q, G, h, A, b


def onehot_qp(n: int = 64, neq: int = 40, *, seed: int = 0, index: int = 0, dtype=np.float32):
    """Structured one-hot QP: Q = 0.1·I, q ~ N(0,1), G = -I, h = 0 (z >= 0),
    A ~ N(0,1) dense neq×n, b = A u with u ~ U[0,1]^n (so u is a feasible point)."""
    r = _rng(seed, WL_ONEHOT, index)
    Q = 0.1 * np.eye(n)
    q = r.standard_normal(n)
    G = -np.eye(n)
    h = np.zeros(n)
    A = r.standard_normal((neq, n))
    u = r.uniform(0.0, 1.0, n)
    Q, q, G, h, A = (_round(x, dtype) for x in (Q, q, G, h, A))
    b = _round(A @ u, dtype)
    return Q, q, G, h, A, b


def psd_qp(n: int, nineq_extra: int, neq: int, rank: int, *, seed: int = 0, index: int = 0,
           dtype=np.float32):
    """A QP with positive semidefinite Q of the given rank (rank 0: a linear program):
    Q = L Lᵀ with L ~ N(0,1)/√n (n × rank), q ~ N(0,1), the box −1 ≤ z ≤ 1 plus nineq_extra
    rows G ~ N(0,1) with h = G z0 + s0 (z0 ~ U(−0.3, 0.3), s0 ~ U(0.2, 1)), A ~ N(0,1), b = A z0,
    so the feasible set is bounded with z0 strictly inside it."""
    r = _rng(seed, WL_PSD, index)
    L = r.standard_normal((n, rank)) / math.sqrt(n)
    Q = L @ L.T
    Q = 0.5 * (Q + Q.T)
    q = r.standard_normal(n)
    Gr = r.standard_normal((nineq_extra, n))
    z0 = r.uniform(-0.3, 0.3, n)
    s0 = r.uniform(0.2, 1.0, nineq_extra)
    A = r.standard_normal((neq, n))
    Q, q, Gr, A, z0 = (_round(x, dtype) for x in (Q, q, Gr, A, z0))
    G = np.vstack([np.eye(n), -np.eye(n), Gr])
    h = np.concatenate([np.ones(2 * n), _round(Gr @ z0 + s0, dtype)])
    b = _round(A @ z0, dtype)
    return Q, q, G, h, A, b


def tv_qp(y, w: float, D=None):
    """Total-variation denoising (§4.2) as a QP in (z, t), FP64:
    minimise ½‖y − z‖² + w·1ᵀt subject to Dz − t ≤ 0 and −Dz − t ≤ 0, with D the first
    difference (n−1)×n unless another operator is given (the learned-D variant).
    Q = diag(I, 0) is positive semidefinite."""
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    D = np.diff(np.eye(n), axis=0) if D is None else np.asarray(D, dtype=np.float64)
    k = D.shape[0]
    Q = np.zeros((n + k, n + k))
    Q[:n, :n] = np.eye(n)
    q = np.concatenate([-y, w * np.ones(k)])
    G = np.block([[D, -np.eye(k)], [-D, -np.eye(k)]])
    h = np.zeros(2 * k)
    return Q, q, G, h, np.zeros((0, n + k)), np.zeros(0)


def tv_signal(n: int, *, seed: int = 0, index: int = 0, noise: float = 0.2) -> np.ndarray:
    """Piecewise-constant signal (3 levels ~ U(−1, 1), random breakpoints) plus N(0, noise²)."""
    r = _rng(seed, WL_TV, index)
    cuts = np.sort(r.choice(np.arange(1, n), 2, replace=False))
    levels = r.uniform(-1.0, 1.0, 3)
    x = np.concatenate([np.full(cuts[0], levels[0]), np.full(cuts[1] - cuts[0], levels[1]),
                        np.full(n - cuts[1], levels[2])])
    return x + noise * r.standard_normal(n)


def stack(instances) -> QPBatch:
    cols = list(zip(*instances))
    return QPBatch(*(np.stack(c) for c in cols))


def random_batch(B: int, n: int, nineq: int, neq: int, *, seed: int = 0,
                 workload: int = WL_SWEEP, dtype=np.float32, start: int = 0) -> QPBatch:
    """B random QPs of one size (instances ``start .. start+B-1`` of the workload stream),
    stored in ``dtype``."""
    inst = [random_qp(n, nineq, neq, seed=seed, workload=workload, index=start + i, dtype=dtype)
            for i in range(B)]
    return stack(inst).astype(dtype)


def onehot_batch(B: int, n: int = 64, neq: int = 40, *, seed: int = 0, dtype=np.float32,
                 start: int = 0) -> QPBatch:
    inst = [onehot_qp(n, neq, seed=seed, index=start + i, dtype=dtype) for i in range(B)]
    return stack(inst).astype(dtype)


def onehot_target(B: int, n: int = 64, *, seed: int = 0, start: int = 0, dtype=np.float32):
    """Random regression target ~ U[0,1]^n for the MSE loss of the one-hot workload."""
    out = np.empty((B, n))
    for i in range(B):
        r = _rng(seed + 7919, WL_ONEHOT, start + i)
        out[i] = r.uniform(0.0, 1.0, n)
    return out.astype(dtype)


def upstream_grad(B: int, n: int, *, seed: int = 0, workload: int = WL_SWEEP, start: int = 0,
                  dtype=np.float32) -> np.ndarray:
    """dℓ/dz* ~ N(0,1), one independent stream per instance."""
    out = np.empty((B, n))
    for i in range(B):
        r = _rng(seed + 104729, workload, start + i)
        out[i] = r.standard_normal(n)
    return out.astype(dtype)


def uneven_sizes(count: int, *, seed: int = 0, n_lo: int = 8, n_hi: int = 256):
    """Per-instance (n, nineq, neq) of the uneven workload: n ~ U{n_lo..n_hi},
    nineq ~ U{n/2..2n}, neq ~ U{0..n/4}."""
    sizes = []
    for i in range(count):
        r = _rng(seed + 31337, WL_UNEVEN, i)
        n = int(r.integers(n_lo, n_hi + 1))
        nineq = int(r.integers(max(1, n // 2), 2 * n + 1))
        neq = int(r.integers(0, n // 4 + 1))
        sizes.append((n, nineq, neq))
    return sizes


def serve_sizes(count: int, *, seed: int = 0, n_lo: int = 16, n_hi: int = 512):
    """Per-request (n, nineq, neq) of the serving stream: n log-uniform in [n_lo, n_hi],
    nineq = n, neq = n/4."""
    sizes = []
    for i in range(count):
        r = _rng(seed + 4242, WL_SERVE, i)
        n = int(round(math.exp(r.uniform(math.log(n_lo), math.log(n_hi)))))
        sizes.append((n, n, n // 4))
    return sizes


def poisson_arrivals(count: int, rate: float, *, seed: int = 0) -> np.ndarray:
    """Arrival times (seconds) of a Poisson stream with the given rate."""
    r = _rng(seed + 99991, WL_SERVE, 0)
    return np.cumsum(r.exponential(1.0 / rate, count))
