"""``QPFunction``: the OptNet QP layer as a ``torch.autograd.Function`` (§3).

forward(Q, q, G, h, A, b) -> z*, λ*, ν*, status.  backward(∂ℓ/∂z*, ∂ℓ/∂λ*, ∂ℓ/∂ν*) -> the
six parameter gradients of Eq. 8, from the factorisation the forward pass left in its
workspace (§3.1.1).  The paper differentiates z* only; λ* and ν* are differentiable here
through the same adjoint with the extra right-hand-side blocks (``qp_backward_ext``).
"""
from __future__ import annotations

import torch

from .qp import ForwardResult, qp_backward, qp_forward


class QPFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q, q, G, h, A, b, options=None):
        fwd = qp_forward(Q, q, G, h, A, b, options=options)
        # Tensors go through save_for_backward (autograd's version checks catch an in-place
        # change of Q, G or A before the backward pass, and no reference cycle keeps the
        # workspace alive); only option and shape metadata stay on ctx.
        ctx.save_for_backward(fwd.Q, fwd.G, fwd.A, fwd.z, fwd.lam, fwd.nu, fwd.workspace)
        ctx.options = fwd.options
        ctx.shapes = (G is None, A is None)
        ctx.mark_non_differentiable(fwd.status)
        ctx.set_materialize_grads(False)   # unused outputs' gradients arrive as None
        return fwd.z, fwd.lam, fwd.nu, fwd.status

    @staticmethod
    def backward(ctx, dz, dlam, dnu, dstatus):
        if dz is None and dlam is None and dnu is None:
            return (None,) * 7
        Qc, Gc, Ac, z, lam, nu, ws = ctx.saved_tensors
        fwd = ForwardResult(z, lam, nu, None, None, None, ws, Qc, Gc, Ac, ctx.options)
        if dz is None:
            dz = torch.zeros_like(z)
        need = ctx.needs_input_grad[:6]
        g = qp_backward(fwd, dz, dl_dlam=dlam, dl_dnu=dnu,
                        need=tuple(bool(x) for x in need))
        no_g, no_a = ctx.shapes
        grads = list(g)
        if no_g:
            grads[2] = grads[3] = None
        if no_a:
            grads[4] = grads[5] = None
        return (*grads, None)


def qp_layer(Q, q, G=None, h=None, A=None, b=None, options=None):
    """z* of the batch, differentiable with respect to every input tensor."""
    z, _, _, _ = QPFunction.apply(Q, q, G, h, A, b, options)
    return z
