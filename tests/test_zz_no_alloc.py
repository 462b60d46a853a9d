"""qp_forward_noalloc: the forward entry point for callers that cannot allocate device memory
(a control loop with a hard latency budget, a process whose device memory is fixed when it
starts, a plugin whose host framework owns all allocation).  Its workspace is the library's
own fixed device array.

Called through the C ABI on two calls in a row with different data and sizes, and compared
with qp_forward: the same kernel on the same data, so the results must be bit-identical.
Around each call, the caching allocator's allocated bytes and the device's free bytes must
not change (outputs are allocated before the call).  This file is collected last."""
import ctypes

import pytest
import torch

from paper_1703_00443_gb300 import _lib, default_options, inputs, qp_forward

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() else None


def _noalloc_call(T, opts, outs):
    lib = _lib.load()
    Q, q, G, h, A, b = T
    B, n, p, m = Q.shape[0], Q.shape[1], G.shape[1], A.shape[1]
    z, lam, nu, st, it = outs
    return lib.qp_forward_noalloc(ctypes.byref(opts), 0, B, n, p, m, *[_ptr(t) for t in T],
                                  _ptr(z), _ptr(lam), _ptr(nu), _ptr(st), _ptr(it), None,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_forward_matches_qp_forward_twice_without_allocating():
    opts = default_options(torch.float32)
    for k, (B, n, p, m) in enumerate([(128, 100, 100, 50), (64, 30, 45, 7)]):
        batch = inputs.random_batch(B, n, p, m, workload=inputs.WL_SWEEP, start=500 * k)
        T = [torch.from_numpy(x).to(DEV) for x in (batch.Q, batch.q, batch.G, batch.h, batch.A, batch.b)]
        outs = (torch.empty((B, n), device=DEV), torch.empty((B, p), device=DEV),
                torch.empty((B, m), device=DEV), torch.empty((B,), device=DEV, dtype=torch.int32),
                torch.empty((B,), device=DEV, dtype=torch.int32))
        torch.cuda.synchronize()
        alloc0, free0 = torch.cuda.memory_allocated(DEV), torch.cuda.mem_get_info(DEV)[0]
        rc = _noalloc_call(T, opts, outs)
        torch.cuda.synchronize()
        assert rc == 0, _lib.load().qp_strerror(rc)
        assert torch.cuda.memory_allocated(DEV) == alloc0
        if k > 0:
            # the first call on the device may load the module that holds the scratch array;
            # after that, a call leaves the device's free memory exactly as it found it
            assert torch.cuda.mem_get_info(DEV)[0] == free0
        ref = qp_forward(*T, options=opts)
        torch.cuda.synchronize()
        z, lam, nu, st, it = outs
        assert torch.equal(st, ref.status) and torch.equal(it, ref.iters)
        for a, r in ((z, ref.z), (lam, ref.lam), (nu, ref.nu)):
            assert torch.equal(a, r)


def test_noalloc_rejects_batches_beyond_its_scratch():
    lib = _lib.load()
    opts = default_options(torch.float32)
    need = lib.qp_workspace_bytes_opt(ctypes.byref(opts), 0, 200, 100, 100, 50)
    assert need > (32 << 20)
    rc = lib.qp_forward_noalloc(ctypes.byref(opts), 0, 200, 100, 100, 50, *([None] * 12), None)
    assert rc == 2   # QP_ENOSPACE, nothing launched
