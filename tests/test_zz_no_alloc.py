"""qp_forward_noalloc, the forward entry point for callers that cannot allocate device memory
(its workspace is the library's own fixed device array).  Called through the C ABI and
compared with qp_forward on two calls in a row with different data."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1703_00443_gb300 import _lib, default_options, inputs, qp_forward
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _noalloc(T, opts):
    lib = _lib.load()
    Q, q, G, h, A, b = T
    B, n, p, m = Q.shape[0], Q.shape[1], G.shape[1], A.shape[1]
    z = torch.empty((B, n), device=DEV)
    lam = torch.empty((B, p), device=DEV)
    nu = torch.empty((B, m), device=DEV)
    st = torch.empty((B,), device=DEV, dtype=torch.int32)
    it = torch.empty((B,), device=DEV, dtype=torch.int32)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t.numel() else None  # noqa: E731
    rc = lib.qp_forward_noalloc(ctypes.byref(opts), 0, B, n, p, m, *[ptr(t) for t in T],
                                ptr(z), ptr(lam), ptr(nu), ptr(st), ptr(it), None,
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, z, lam, nu, st


@pytest.mark.parametrize("sizes", [[(128, 100, 100, 50), (64, 30, 45, 7)]])
def test_noalloc_forward_matches_qp_forward_twice(sizes):
    opts = default_options(torch.float32)
    for k, (B, n, p, m) in enumerate(sizes):
        batch = inputs.random_batch(B, n, p, m, workload=inputs.WL_SWEEP, start=500 * k)
        T = [torch.from_numpy(x).to(DEV) for x in (batch.Q, batch.q, batch.G, batch.h, batch.A, batch.b)]
        rc, z, lam, nu, st = _noalloc(T, opts)
        assert rc == 0, _lib.load().qp_strerror(rc)
        ref = qp_forward(*T, options=opts)
        torch.cuda.synchronize()
        assert torch.equal(st, ref.status)
        for a, r in ((z, ref.z), (lam, ref.lam), (nu, ref.nu)):
            assert rel_err(a.double().cpu().numpy(), r.double().cpu().numpy()).max() <= 1e-5


def test_noalloc_rejects_batches_beyond_its_scratch():
    lib = _lib.load()
    opts = default_options(torch.float32)
    need = lib.qp_workspace_bytes_opt(ctypes.byref(opts), 0, 200, 100, 100, 50)
    assert need > (32 << 20)
    rc = lib.qp_forward_noalloc(ctypes.byref(opts), 0, 200, 100, 100, 50, *([None] * 12), None)
    assert rc == 2   # QP_ENOSPACE, nothing launched
