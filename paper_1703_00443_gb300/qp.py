"""Python binding of the C ABI (argument marshalling only; every step runs in the CUDA
library).  PyTorch provides device memory and the stream.

    fwd = qp_forward(Q, q, G, h, A, b)             # z*, λ*, ν*, status, iters, workspace
    grads = qp_backward(fwd, dl_dz)                 # dQ, dq, dG, dh, dA, db

Shapes (batch-major, row-major, contiguous CUDA tensors of one dtype, float32 or float64):
Q [B,n,n], q [B,n], G [B,nineq,n], h [B,nineq], A [B,neq,n], b [B,neq].  G/h or A/b may be
None (or have zero rows) when there are no inequality or equality constraints.
"""
from __future__ import annotations

import ctypes
import dataclasses

import torch

from . import _lib

QP_F32, QP_F64 = 0, 1
STATUS_CONVERGED, STATUS_MAX_ITER, STATUS_NOT_PD, STATUS_NUMERICAL = 0, 1, 2, 3
STATUS_NO_FORWARD, STATUS_INFEASIBLE, STATUS_TIMEOUT = 4, 5, 6
FLAG_NEAR_DEGENERATE = 0x100   # in backward status words (status & 0xff is the code)
FLAG_REGULARIZED_Q = 0x200     # backward status word: Q was singular, Q + δI was factored


class QPError(RuntimeError):
    pass


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return QP_F32
    if t.dtype == torch.float64:
        return QP_F64
    raise QPError(f"unsupported dtype {t.dtype}; use float32 or float64")


def _check(rc: int):
    if rc != 0:
        lib = _lib.load()
        raise QPError(f"qp call failed ({rc}): {lib.qp_strerror(rc).decode()}")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def default_options(dtype=torch.float32) -> _lib.QPOptions:
    lib = _lib.load()
    o = _lib.QPOptions()
    lib.qp_default_options(QP_F32 if dtype == torch.float32 else QP_F64, ctypes.byref(o))
    return o


def workspace_bytes(dtype, B, n, nineq, neq) -> int:
    lib = _lib.load()
    return int(lib.qp_workspace_bytes(QP_F32 if dtype == torch.float32 else QP_F64, B, n, nineq, neq))


def supported(dtype, n, nineq, neq) -> bool:
    lib = _lib.load()
    return lib.qp_supported(QP_F32 if dtype == torch.float32 else QP_F64, n, nineq, neq) == 0


def _prep(Q, q, G, h, A, b):
    if Q.dim() != 3 or Q.shape[1] != Q.shape[2]:
        raise QPError("Q must be [B, n, n]")
    B, n = Q.shape[0], Q.shape[1]
    dev, dt = Q.device, Q.dtype
    if dev.type != "cuda":
        raise QPError("tensors must live on a CUDA device (there is no CPU path)")
    if G is None or G.numel() == 0:
        G = torch.empty((B, 0, n), device=dev, dtype=dt)
        h = torch.empty((B, 0), device=dev, dtype=dt)
    if A is None or A.numel() == 0:
        A = torch.empty((B, 0, n), device=dev, dtype=dt)
        b = torch.empty((B, 0), device=dev, dtype=dt)
    out = []
    for name, t, shape in (("Q", Q, (B, n, n)), ("q", q, (B, n)), ("G", G, (B, G.shape[1], n)),
                           ("h", h, (B, G.shape[1])), ("A", A, (B, A.shape[1], n)),
                           ("b", b, (B, A.shape[1]))):
        if tuple(t.shape) != shape:
            raise QPError(f"{name} has shape {tuple(t.shape)}, expected {shape}")
        if t.device != dev or t.dtype != dt:
            raise QPError(f"{name} must be on {dev} with dtype {dt}")
        out.append(t.contiguous())
    return out


@dataclasses.dataclass
class ForwardResult:
    z: torch.Tensor
    lam: torch.Tensor
    nu: torch.Tensor
    status: torch.Tensor
    iters: torch.Tensor
    resid: torch.Tensor
    workspace: torch.Tensor
    Q: torch.Tensor
    G: torch.Tensor
    A: torch.Tensor
    options: _lib.QPOptions


def alloc_workspace(dtype, B, n, nineq, neq, device, options=None) -> torch.Tensor:
    if options is None:
        nbytes = workspace_bytes(dtype, B, n, nineq, neq)
    else:
        lib = _lib.load()
        nbytes = int(lib.qp_workspace_bytes_opt(ctypes.byref(options),
                                                QP_F32 if dtype == torch.float32 else QP_F64,
                                                B, n, nineq, neq))
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def uses_global_path(dtype, n, nineq, neq) -> bool:
    lib = _lib.load()
    return lib.qp_uses_global_path(QP_F32 if dtype == torch.float32 else QP_F64, n, nineq, neq) == 1


def uses_tensor_cores(dtype, n, nineq, neq, options=None) -> bool:
    """Whether the setup factorisation of this size runs on the tensor cores."""
    lib = _lib.load()
    opt = ctypes.byref(options) if options is not None else None
    return lib.qp_uses_tensor_cores(opt, QP_F32 if dtype == torch.float32 else QP_F64,
                                    n, nineq, neq) == 1


def qp_forward(Q, q, G=None, h=None, A=None, b=None, *, options=None, workspace=None,
               out=None) -> ForwardResult:
    """Solve the batch (C ABI ``qp_forward``) on the current CUDA stream."""
    Q, q, G, h, A, b = _prep(Q, q, G, h, A, b)
    B, n, nineq, neq = Q.shape[0], Q.shape[1], G.shape[1], A.shape[1]
    dev, dt = Q.device, Q.dtype
    code = _dtype_code(Q)
    lib = _lib.load()
    opts = options if options is not None else default_options(dt)
    if workspace is None:
        workspace = alloc_workspace(dt, B, n, nineq, neq, dev, opts)
    if out is None:
        z = torch.empty((B, n), device=dev, dtype=dt)
        lam = torch.empty((B, nineq), device=dev, dtype=dt)
        nu = torch.empty((B, neq), device=dev, dtype=dt)
        status = torch.empty((B,), device=dev, dtype=torch.int32)
        iters = torch.empty((B,), device=dev, dtype=torch.int32)
        resid = torch.empty((B, 4), device=dev, dtype=torch.float64)
    else:
        z, lam, nu, status, iters = out[:5]
        resid = out[5] if len(out) > 5 else None
    with torch.cuda.device(dev):
        rc = lib.qp_forward(ctypes.byref(opts), code, B, n, nineq, neq,
                            _ptr(Q), _ptr(q), _ptr(G), _ptr(h), _ptr(A), _ptr(b),
                            _ptr(z), _ptr(lam), _ptr(nu), _ptr(status), _ptr(iters),
                            _ptr(resid), _ptr(workspace), workspace.numel(), _stream_handle(dev))
    _check(rc)
    return ForwardResult(z, lam, nu, status, iters, resid, workspace, Q, G, A, opts)


def qp_backward(fwd: ForwardResult, dl_dz: torch.Tensor, *, dl_dlam=None, dl_dnu=None,
                need=(True,) * 6, options=None, out=None, status=None):
    """Gradients (dQ, dq, dG, dh, dA, db) of ℓ(z*) (C ABI ``qp_backward``), or of ℓ(z*, λ*, ν*)
    when ``dl_dlam`` ([B, nineq]) or ``dl_dnu`` ([B, neq]) is given (``qp_backward_ext``);
    entries for which ``need`` is False come back as None.  ``status``: an int32 [B] CUDA
    tensor that receives each instance's backward status word (forward status code, or
    STATUS_NO_FORWARD when the workspace holds no matching forward pass; flag bits above the
    low 8, e.g. FLAG_NEAR_DEGENERATE)."""
    Q, G, A = fwd.Q, fwd.G, fwd.A
    B, n, nineq, neq = Q.shape[0], Q.shape[1], G.shape[1], A.shape[1]
    dev, dt = Q.device, Q.dtype
    dl_dz = dl_dz.to(device=dev, dtype=dt).contiguous()
    if tuple(dl_dz.shape) != (B, n):
        raise QPError(f"dl_dz has shape {tuple(dl_dz.shape)}, expected {(B, n)}")
    lib = _lib.load()
    opts = options if options is not None else fwd.options
    shapes = [(B, n, n), (B, n), (B, nineq, n), (B, nineq), (B, neq, n), (B, neq)]
    if out is None:
        grads = [torch.empty(s, device=dev, dtype=dt) if w else None for s, w in zip(shapes, need)]
    else:
        grads = list(out)
    extra = []
    for name, t, k in (("dl_dlam", dl_dlam, nineq), ("dl_dnu", dl_dnu, neq)):
        if t is not None:
            t = t.to(device=dev, dtype=dt).contiguous()
            if tuple(t.shape) != (B, k):
                raise QPError(f"{name} has shape {tuple(t.shape)}, expected {(B, k)}")
        extra.append(t if t is not None and t.numel() else None)
    if status is not None and (status.dtype != torch.int32 or status.device != dev
                               or status.numel() < B or not status.is_contiguous()):
        raise QPError("status must be a contiguous int32 tensor of B elements on the device")
    with torch.cuda.device(dev):
        if extra[0] is None and extra[1] is None and status is None:
            rc = lib.qp_backward(ctypes.byref(opts), _dtype_code(Q), B, n, nineq, neq,
                                 _ptr(Q), _ptr(G), _ptr(A), _ptr(fwd.workspace),
                                 fwd.workspace.numel(), _ptr(dl_dz),
                                 *[_ptr(g) for g in grads], _stream_handle(dev))
        else:
            rc = lib.qp_backward_ext(ctypes.byref(opts), _dtype_code(Q), B, n, nineq, neq,
                                     _ptr(Q), _ptr(G), _ptr(A), _ptr(fwd.workspace),
                                     fwd.workspace.numel(), _ptr(dl_dz), _ptr(extra[0]),
                                     _ptr(extra[1]), *[_ptr(g) for g in grads], _ptr(status),
                                     _stream_handle(dev))
    _check(rc)
    return tuple(grads)
