"""Packed batches of QPs of uneven sizes (C ABI ``qp_packed_plan`` / ``qp_forward_packed`` /
``qp_backward_packed``): one persistent launch per direction, each instance on the kernel path
its own size selects, the work queue ordered largest estimated cost first.

    pb = PackedBatch([(n0, nineq0, neq0), (n1, nineq1, neq1), ...])
    Qp, qp, Gp, hp, Ap, bp = pb.pack(instances)        # flat device tensors
    out = pb.forward(Qp, qp, Gp, hp, Ap, bp)           # flat z, λ, ν + status/iters/resid
    grads = pb.backward(pb.pack_vec(dl_dz_list, "q"))  # flat dQ, dq, dG, dh, dA, db
    pb.unpack(out.z, "q")                              # list of per-instance z
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np
import torch

from . import _lib
from .qp import QP_F32, QP_F64, QPError, _check, _ptr, _stream_handle, default_options


@dataclasses.dataclass
class PackedForward:
    z: torch.Tensor
    lam: torch.Tensor
    nu: torch.Tensor
    status: torch.Tensor
    iters: torch.Tensor
    resid: torch.Tensor


class PackedBatch:
    """Plan, workspace and descriptors of one batch composition (reusable across calls and
    safe to capture in a CUDA graph once built)."""

    KEYS = ("Q", "q", "G", "h", "A", "b")

    def __init__(self, dims, dtype=torch.float32, device="cuda", options=None, tuning=None):
        self.dims = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(-1, 3))
        self.B = self.dims.shape[0]
        self.dtype = dtype
        self.device = torch.device(device)
        self.code = QP_F32 if dtype == torch.float32 else QP_F64
        self.options = options if options is not None else default_options(dtype)
        lib = _lib.load()
        self.desc_host = (_lib.QPInstanceDesc * max(self.B, 1))()
        self.sizes = _lib.QPPackedSizes()
        hints = cost = None
        if tuning is not None:
            # per-instance kernel path and predicted time from a measured tuning table
            hints, cost = tuning.plan_arrays(self.dims)
        rc = lib.qp_packed_plan_ex(ctypes.byref(self.options), self.code, self.B,
                                   self.dims.ctypes.data_as(ctypes.c_void_p),
                                   None if hints is None else hints.ctypes.data_as(ctypes.c_void_p),
                                   None if cost is None else cost.ctypes.data_as(ctypes.c_void_p),
                                   self.desc_host, ctypes.byref(self.sizes))
        _check(rc)
        raw = bytes(memoryview(self.desc_host))[: self.B * ctypes.sizeof(_lib.QPInstanceDesc)]
        self.desc = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(self.device) \
            if self.B else torch.empty(0, dtype=torch.uint8, device=self.device)
        self.workspace = torch.empty(max(int(self.sizes.ws_bytes), 256), dtype=torch.uint8,
                                     device=self.device)
        # per-instance offsets in index order (the descriptor array is in execution order)
        self.offsets = {}
        order = sorted(range(self.B), key=lambda k: self.desc_host[k].id)
        for key, fld in (("Q", "oQ"), ("q", "oq"), ("G", "oG"), ("h", "oh"), ("A", "oA"),
                         ("b", "ob")):
            self.offsets[key] = np.array([getattr(self.desc_host[k], fld) for k in order],
                                         dtype=np.int64)
        n, p, m = self.dims[:, 0].astype(np.int64), self.dims[:, 1].astype(np.int64), \
            self.dims[:, 2].astype(np.int64)
        self.lengths = {"Q": n * n, "q": n, "G": p * n, "h": p, "A": m * n, "b": m}
        self.shapes = {"Q": list(zip(n, n)), "q": list(zip(n)), "G": list(zip(p, n)),
                       "h": list(zip(p)), "A": list(zip(m, n)), "b": list(zip(m))}
        self.totals = {"Q": int(self.sizes.nQ), "q": int(self.sizes.nq), "G": int(self.sizes.nG),
                       "h": int(self.sizes.nh), "A": int(self.sizes.nA), "b": int(self.sizes.nb)}
        self.n_global = int(self.sizes.n_global)

    # ---------------------------------------------------------------- packing helpers
    def pack_vec(self, items, key):
        """Place per-instance arrays (any shape, row-major) at their planned offsets in a flat
        buffer for ``key`` (offsets are padded to 4 elements; the gaps hold zeros)."""
        out = torch.zeros(max(self.totals[key], 1), dtype=self.dtype, device=self.device)
        items = list(items)
        if len(items) != self.B:
            raise QPError(f"{len(items)} items for {self.B} instances")
        for o, l, x in zip(self.offsets[key], self.lengths[key], items):
            t = torch.as_tensor(x).reshape(-1)
            if t.numel() != l:
                raise QPError(f"{key}: instance has {t.numel()} elements, expected {l}")
            if l:
                out[o:o + l] = t.to(device=self.device, dtype=self.dtype)
        return out

    def pack(self, instances):
        """instances: list of (Q, q, G, h, A, b) arrays/tensors of the planned sizes."""
        cols = list(zip(*instances))
        return tuple(self.pack_vec(c, k) for c, k in zip(cols, self.KEYS))

    def unpack(self, flat, key):
        offs, lens, shp = self.offsets[key], self.lengths[key], self.shapes[key]
        return [flat[o:o + l].view(*s) for o, l, s in zip(offs, lens, shp)]

    # ---------------------------------------------------------------- calls
    def _buf(self, t):
        return None if t is None or t.numel() == 0 else t

    def forward(self, Q, q, G, h, A, b, out=None) -> PackedForward:
        lib = _lib.load()
        dev = self.device
        if out is None:   # zero-filled so the padding gaps between instances are defined
            z = torch.zeros(max(self.totals["q"], 1), dtype=self.dtype, device=dev)
            lam = torch.zeros(max(self.totals["h"], 1), dtype=self.dtype, device=dev)
            nu = torch.zeros(max(self.totals["b"], 1), dtype=self.dtype, device=dev)
            status = torch.empty(max(self.B, 1), dtype=torch.int32, device=dev)
            iters = torch.empty(max(self.B, 1), dtype=torch.int32, device=dev)
            resid = torch.empty((max(self.B, 1), 4), dtype=torch.float64, device=dev)
            out = PackedForward(z, lam, nu, status, iters, resid)
        with torch.cuda.device(dev):
            rc = lib.qp_forward_packed(
                ctypes.byref(self.options), self.code, self.B,
                ctypes.c_void_p(self.desc.data_ptr()), ctypes.byref(self.sizes),
                _ptr(Q), _ptr(q), _ptr(self._buf(G)), _ptr(self._buf(h)), _ptr(self._buf(A)),
                _ptr(self._buf(b)), _ptr(out.z), _ptr(out.lam), _ptr(out.nu), _ptr(out.status),
                _ptr(out.iters), _ptr(out.resid), _ptr(self.workspace), self.workspace.numel(),
                _stream_handle(dev))
        _check(rc)
        return out

    def backward(self, Q, G, A, dl_dz, out=None, status=None):
        """Gradients packed like the inputs; ``status`` (int32 [B] CUDA tensor, by instance
        index) receives each instance's backward status word when given."""
        lib = _lib.load()
        dev = self.device
        if out is None:
            out = tuple(torch.zeros(max(self.totals[k], 1), dtype=self.dtype, device=dev)
                        for k in self.KEYS)
        with torch.cuda.device(dev):
            rc = lib.qp_backward_packed(
                ctypes.byref(self.options), self.code, self.B,
                ctypes.c_void_p(self.desc.data_ptr()), ctypes.byref(self.sizes),
                _ptr(Q), _ptr(self._buf(G)), _ptr(self._buf(A)), _ptr(self.workspace),
                self.workspace.numel(), _ptr(dl_dz), *[_ptr(g) for g in out], _ptr(status),
                _stream_handle(dev))
        _check(rc)
        return out
