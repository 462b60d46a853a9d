"""Tuning-table logic without a GPU: the fit recovers a planted cost model and the planner
hints follow the predictions and the feasibility of the shared-memory path."""
import numpy as np

from paper_1703_00443_gb300 import autotune
from paper_1703_00443_gb300.autotune import Tuning, features, fit


def test_fit_recovers_planted_model():
    true = {"smem": np.array([2e-12, 5e-10, 1e-9, 1e-4]), "global": np.array([6e-12, 9e-10, 2e-9, 2e-4])}
    rows = []
    for (n, p, m) in autotune.default_classes():
        for path in ("smem", "global"):
            rows.append({"n": n, "nineq": p, "neq": m, "path": path,
                         "seconds": float(true[path] @ features(n, p, m, path))})
    coef = fit(rows)
    for path in true:
        np.testing.assert_allclose(coef[path], true[path], rtol=1e-6)


def test_plan_arrays_prefers_faster_feasible_path():
    # global path 10x cheaper in this planted table -> always chosen
    t = Tuning({"smem": [1e-10, 0, 0, 1e-3], "global": [1e-11, 0, 0, 1e-4]})
    hints, cost = t.plan_arrays([(10, 10, 2), (400, 400, 100)])
    assert list(hints) == [1, 1] and cost.dtype == np.float32 and (cost > 0).all()
    # shared-memory path cheaper: chosen where it can run, global elsewhere
    t = Tuning({"smem": [1e-12, 0, 0, 1e-5], "global": [1e-10, 0, 0, 1e-3]})
    hints, _ = t.plan_arrays([(10, 10, 2), (400, 400, 100)])
    assert list(hints) == [2, 1]


def test_roundtrip_json(tmp_path):
    t = Tuning({"smem": [1, 2, 3, 4], "global": [5, 6, 7, 8]}, [{"n": 1}])
    p = tmp_path / "t.json"
    t.save(str(p))
    u = Tuning.load(str(p))
    assert np.allclose(u.coef["global"], [5, 6, 7, 8]) and u.measurements == [{"n": 1}]
