"""Closed-form QP layers of the paper's appendix (tests/golden/closed_forms.json, written by
tests/golden/make_closed_forms.py from the closed forms alone): ReLU (Eq. 21), sum of
maxima (Eq. 19), the three-term maximum (Eq. 24) and the simplex projection (Eq. 25), with
the gradient ∂ℓ/∂q where the closed form gives it.  The oracle must reproduce them (CPU),
and so must the CUDA path through the C ABI, in FP64 and FP32 (GPU), without the oracle."""
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
CASES = json.load(open(os.path.join(HERE, "golden", "closed_forms.json")))["cases"]


def _arrays(c):
    n, p, m = c["n"], c["nineq"], c["neq"]
    f = lambda k, *shape: np.array(c[k], dtype=np.float64).reshape(*shape)  # noqa: E731
    return (f("Q", n, n), f("q", n), f("G", p, n), f("h", p), f("A", m, n), f("b", m))


@pytest.mark.parametrize("c", CASES, ids=[c["name"] for c in CASES])
def test_oracle_reproduces_closed_forms(c):
    Q, q, G, h, A, b = _arrays(c)
    sol = oracle.solve(Q, q, G, h, A, b)
    z = np.array(c["z"])
    assert np.abs(sol["z"] - z).max() <= 1e-9 * max(1.0, np.abs(z).max())
    if "dq" in c:
        gr = oracle.backward(Q, G, h, A, sol, np.array(c["dl_dz"]))
        assert np.abs(gr["dq"] - np.array(c["dq"])).max() <= 1e-8 * max(1.0, np.abs(c["dq"]).max())


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("c", CASES, ids=[c["name"] for c in CASES])
def test_cuda_path_reproduces_closed_forms(c, dtype):
    import torch

    from paper_1703_00443_gb300 import qp_backward, qp_forward
    tdt = torch.float64 if dtype == "f64" else torch.float32
    ztol, gtol = (1e-9, 1e-8) if dtype == "f64" else (1e-5, 1e-4)
    T = [torch.from_numpy(x).to(tdt).unsqueeze(0).to("cuda:0") for x in _arrays(c)]
    fwd = qp_forward(*T)
    torch.cuda.synchronize()
    assert int(fwd.status[0]) == 0, int(fwd.status[0])
    z = np.array(c["z"])
    zg = fwd.z[0].double().cpu().numpy()
    assert np.abs(zg - z).max() <= ztol * max(1.0, np.abs(z).max()), np.abs(zg - z).max()
    if "dq" in c:
        g = torch.tensor(c["dl_dz"], dtype=tdt, device="cuda:0").unsqueeze(0)
        grads = qp_backward(fwd, g)
        dq = grads[1][0].double().cpu().numpy()
        ref = np.array(c["dq"])
        scale = max(np.abs(ref).max(), 1e-3 * np.abs(c["dl_dz"]).max())
        assert np.abs(dq - ref).max() <= gtol * scale, np.abs(dq - ref).max()
