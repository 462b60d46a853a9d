"""QPFunction (autograd) against the FP64 oracle and against central finite differences."""
import numpy as np
import pytest
import torch

from paper_1703_00443_gb300 import QPFunction, inputs, qp_layer
from tests.helpers import grad_floor, oracle_solve_and_grad, rel_err

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_autograd_matches_oracle_gradients():
    B, n, p, m = 6, 20, 20, 10
    batch = inputs.random_batch(B, n, p, m, workload=inputs.WL_SWEEP, dtype=np.float32, start=50)
    g = inputs.upstream_grad(B, n, start=50)
    T = [torch.from_numpy(x).to(DEV).requires_grad_(True) for x in
         (batch.Q, batch.q, batch.G, batch.h, batch.A, batch.b)]
    z = qp_layer(*T)
    (z * torch.from_numpy(g).to(DEV)).sum().backward()
    sols, grads = oracle_solve_and_grad(batch, g)
    for t, name in zip(T, ("dQ", "dq", "dG", "dh", "dA", "db")):
        fl = grad_floor(name, g, [s["z"] for s in sols])
        e = rel_err(t.grad.double().cpu().numpy(), [gr[name] for gr in grads], fl)
        assert e.max() <= 1e-4, (name, e.max())


def test_gradcheck_fp64_central_differences():
    """torch.autograd.gradcheck compares the adjoint gradients with central differences of
    the FP64 solve (Q perturbed symmetrically through a symmetric parametrisation)."""
    n, p, m = 4, 6, 1
    batch = inputs.random_batch(2, n, p, m, workload=inputs.WL_PLAIN, dtype=np.float64, start=77)
    Q0, q, G, h, A, b = (torch.from_numpy(x).to(DEV) for x in
                         (batch.Q, batch.q, batch.G, batch.h, batch.A, batch.b))
    q = (2.0 * q).requires_grad_(True)
    Lq = torch.linalg.cholesky(Q0).requires_grad_(True)
    G.requires_grad_(True)
    h.requires_grad_(True)
    A.requires_grad_(True)
    b.requires_grad_(True)

    def f(Lq, q, G, h, A, b):
        Q = Lq @ Lq.transpose(1, 2)
        return qp_layer(Q, q, G, h, A, b)

    assert torch.autograd.gradcheck(f, (Lq, q, G, h, A, b), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_no_constraint_tensors_give_none_grads():
    n = 8
    batch = inputs.random_batch(2, n, 0, 0, workload=inputs.WL_PLAIN, dtype=np.float32)
    Q = torch.from_numpy(batch.Q).to(DEV).requires_grad_(True)
    q = torch.from_numpy(batch.q).to(DEV).requires_grad_(True)
    z = qp_layer(Q, q)
    z.sum().backward()
    ref = -torch.linalg.solve(Q.detach().double(), q.detach().double().unsqueeze(-1)).squeeze(-1)
    assert torch.allclose(z.double(), ref, rtol=1e-5, atol=1e-6)
    assert q.grad is not None and Q.grad is not None


def test_gradcheck_fp64_through_lambda_and_nu():
    """λ* and ν* as differentiable outputs (the adjoint's extra right-hand-side blocks):
    gradcheck against central differences of the FP64 solve."""
    from paper_1703_00443_gb300.autograd import QPFunction
    n, p, m = 4, 6, 1
    batch = inputs.random_batch(2, n, p, m, workload=inputs.WL_PLAIN, dtype=np.float64, start=77)
    Q, q, G, h, A, b = (torch.from_numpy(x).to(DEV) for x in
                        (batch.Q, batch.q, batch.G, batch.h, batch.A, batch.b))
    q = (2.0 * q).requires_grad_(True)
    h.requires_grad_(True)
    b.requires_grad_(True)

    def f(q_, h_, b_):
        z, lam, nu, _ = QPFunction.apply(Q, q_, G, h_, A, b_)
        return z, lam, nu

    assert torch.autograd.gradcheck(f, (q, h, b), eps=1e-6, atol=1e-6, rtol=1e-5)
