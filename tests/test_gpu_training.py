"""End-to-end training through the QP layer on synthetic data: a Sudoku-shaped layer
(n = 64, z ≥ 0, 40 learned equality constraints, §4.4) recovers a hidden constraint matrix
from (input, z*) pairs; the MSE drops and every step's gradients are finite."""
import numpy as np
import pytest
import torch

from paper_1703_00443_gb300 import inputs
from paper_1703_00443_gb300.layers import LearnedEqualityQP

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_learned_equality_layer_trains():
    torch.manual_seed(0)
    n, neq, B = 64, 40, 32
    bt = inputs.onehot_batch(1, n, neq, dtype=np.float64)
    A_true = torch.from_numpy(bt.A[0]).to(DEV, torch.float32)
    u = torch.from_numpy(np.random.default_rng(1).uniform(0.2, 1.0, n)).to(DEV, torch.float32)
    true_layer = LearnedEqualityQP(n, neq, A_true, u).to(DEV)
    A0 = A_true + 0.3 * torch.randn(neq, n, device=DEV)
    layer = LearnedEqualityQP(n, neq, A0, u).to(DEV)
    opt = torch.optim.Adam(layer.parameters(), lr=1e-2)
    p = torch.randn(B, n, device=DEV)
    with torch.no_grad():
        target = true_layer(p)
    losses = []
    for _ in range(40):
        opt.zero_grad()
        loss = torch.nn.functional.mse_loss(layer(p), target)
        loss.backward()
        assert torch.isfinite(layer.A.grad).all()
        opt.step()
        losses.append(loss.item())
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.5 * losses[0], losses[::8]
