"""A QP layer with learned equality constraints, the shape of the paper's Sudoku layer (§4.4).

z*(p) = argmin_z ½ zᵀQz + pᵀz  s.t.  A z = b,  z ≥ 0, with p the layer input (one row per
example), Q = 0.1·I fixed, and A learned.  As in the paper's Sudoku layer the equality
constraints are the parameters; b = A u for a fixed u > 0 keeps every QP feasible (z = u)
while A moves.  The layer runs the batched solver forward and its adjoint backward
(``qp_layer``), so A receives the batch-summed gradient of Eq. 8.
"""
from __future__ import annotations

import torch

from .autograd import qp_layer


class LearnedEqualityQP(torch.nn.Module):
    def __init__(self, n: int, neq: int, A0: torch.Tensor, u: torch.Tensor, q_scale: float = 0.1):
        super().__init__()
        self.n, self.neq = n, neq
        self.A = torch.nn.Parameter(A0.detach().clone())
        self.register_buffer("u", u.detach().clone())
        self.register_buffer("Q", q_scale * torch.eye(n, dtype=A0.dtype, device=A0.device))
        self.register_buffer("G", -torch.eye(n, dtype=A0.dtype, device=A0.device))

    def forward(self, p: torch.Tensor) -> torch.Tensor:
        B = p.shape[0]
        Q = self.Q.expand(B, self.n, self.n)
        G = self.G.expand(B, self.n, self.n)
        h = torch.zeros((B, self.n), dtype=p.dtype, device=p.device)
        A = self.A.expand(B, self.neq, self.n)
        b = (self.A @ self.u).expand(B, self.neq)
        return qp_layer(Q.contiguous(), p, G.contiguous(), h, A.contiguous(), b.contiguous())
