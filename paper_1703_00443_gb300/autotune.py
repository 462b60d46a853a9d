"""Measured tuning of the packed-batch schedule: which kernel path each size takes and the
cost model that orders the persistent work queue.

``measure`` times one wave of instances (one block per SM, so the time is one instance's
latency) for a grid of size classes on every kernel path that can take them; ``fit`` fits,
per path, time ≈ c·[sweep FMAs, per-iteration Schur FMAs, residual FMAs, 1] by least squares;
``Tuning.plan_arrays`` then picks, for each instance of a packed batch, the path with the
smaller predicted time (where both are possible) and hands the predicted times to the
planner, which orders the work queue largest first.  ``autotune`` runs all three and saves
the table as JSON (by default next to the built library).
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import _lib

DEFAULT_PATH = os.path.join(_lib.BUILD, "autotune.json")
PATHS = ("smem", "global")


def padded_nz(n, m, block):
    return n + (block - (n + m) % block) % block


def features(n, p, m, path):
    """Work features of one instance on a path: setup-sweep FMAs, per-iteration Schur
    factorisation FMAs, per-iteration residual FMAs, 1."""
    nz = padded_nz(n, m, 4 if path == "smem" else 16)
    m1 = nz + m
    N = m1 + p
    return np.array([m1 * N * N, p ** 3 / 3.0, N * n, 1.0], dtype=np.float64)


def smem_possible(n, p, m, dtype=torch.float32):
    lib = _lib.load()
    return lib.qp_uses_global_path(0 if dtype == torch.float32 else 1, n, p, m) == 0


class Tuning:
    def __init__(self, coef: dict, measurements=None):
        self.coef = {k: np.asarray(v, dtype=np.float64) for k, v in coef.items()}
        self.measurements = measurements or []

    def predict(self, n, p, m, path):
        return float(max(self.coef[path] @ features(n, p, m, path), 1e-6))

    def choose(self, n, p, m):
        if smem_possible(n, p, m) and self.predict(n, p, m, "smem") <= self.predict(n, p, m, "global"):
            return "smem"
        return "global"

    def plan_arrays(self, dims):
        """int8 path hints (2 shared-memory, 1 global-memory) and float32 predicted times."""
        dims = np.asarray(dims).reshape(-1, 3)
        hints = np.empty(len(dims), dtype=np.int8)
        cost = np.empty(len(dims), dtype=np.float32)
        for i, (n, p, m) in enumerate(dims):
            path = self.choose(int(n), int(p), int(m))
            hints[i] = 2 if path == "smem" else 1
            cost[i] = self.predict(int(n), int(p), int(m), path)
        return hints, cost

    def to_json(self):
        return {"version": 1, "coef": {k: v.tolist() for k, v in self.coef.items()},
                "measurements": self.measurements}

    def save(self, path=DEFAULT_PATH):
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as fh:
            json.dump(self.to_json(), fh, indent=1)

    @classmethod
    def load(cls, path=DEFAULT_PATH):
        with open(path) as fh:
            d = json.load(fh)
        return cls(d["coef"], d.get("measurements"))


def default_classes():
    out = []
    for n in (8, 16, 32, 64, 96, 128, 192, 256):
        for rp in (0.5, 1.0, 2.0):
            for rm in (0.0, 0.25):
                out.append((n, max(1, int(rp * n)), int(rm * n)))
    return out


def measure(classes=None, device="cuda:0", reps=3, distinct=8, seed=0):
    """Per-instance fwd+bwd latency (s) of each class on each possible path."""
    from . import inputs
    from .qp import default_options, qp_backward, qp_forward
    classes = classes or default_classes()
    dev = torch.device(device)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    rows = []
    for (n, p, m) in classes:
        base = inputs.random_batch(distinct, n, p, m, workload=inputs.WL_UNEVEN, seed=seed + 17)
        reps_idx = np.arange(nsm) % distinct
        T = [torch.from_numpy(np.ascontiguousarray(x[reps_idx])).to(dev)
             for x in (base.Q, base.q, base.G, base.h, base.A, base.b)]
        g = torch.from_numpy(inputs.upstream_grad(distinct, n, seed=seed + 17)[reps_idx]).to(dev)
        for path in PATHS:
            if path == "smem" and not smem_possible(n, p, m):
                continue
            o = default_options(torch.float32)
            o.path = 0 if path == "smem" else 1
            f = qp_forward(*T, options=o)
            qp_backward(f, g)
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                f = qp_forward(*T, options=o, workspace=f.workspace)
                qp_backward(f, g)
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1) / 1e3)
            rows.append({"n": n, "nineq": p, "neq": m, "path": path, "seconds": float(np.median(ts)),
                         "iters": float(f.iters.float().mean())})
    return rows


def fit(rows):
    """Least-squares coefficients of the feature model per path (non-negative by clipping)."""
    coef = {}
    for path in PATHS:
        sel = [r for r in rows if r["path"] == path]
        if not sel:
            coef[path] = np.array([0.0, 0.0, 0.0, 1.0])
            continue
        X = np.stack([features(r["n"], r["nineq"], r["neq"], path) for r in sel])
        y = np.array([r["seconds"] for r in sel])
        # relative least squares (weights 1/y) so small instances are fitted too
        w = 1.0 / np.maximum(y, 1e-9)
        c, *_ = np.linalg.lstsq(X * w[:, None], y * w, rcond=None)
        coef[path] = np.maximum(c, 0.0)
    return coef


def autotune(device="cuda:0", classes=None, save_to=DEFAULT_PATH):
    rows = measure(classes, device)
    tun = Tuning(fit(rows), rows)
    if save_to:
        tun.save(save_to)
    return tun
