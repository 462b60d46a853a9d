"""The C-ABI library builds, loads and exports every symbol include/qp_gb300.h declares.
Only host-side entry points are called (no kernel launch needs a GPU here)."""
import ctypes
import os
import re

from paper_1703_00443_gb300 import _lib

HEADER = os.path.join(_lib.INCLUDE, "qp_gb300.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qp_[a-z0-9_]+)\s*\(", text)))


def test_header_declarations_are_exported():
    lib = _lib.load()
    names = declared_functions()
    assert {"qp_forward", "qp_backward", "qp_workspace_bytes"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(_lib.EXPORTS), "binding does not declare every header symbol"


def test_host_side_queries():
    lib = _lib.load()
    o = _lib.QPOptions()
    lib.qp_default_options(0, ctypes.byref(o))
    assert o.max_iter == 50 and o.refine == 4 and o.path == 0 and 0 < o.tol < 1e-6
    lib.qp_default_options(1, ctypes.byref(o))
    assert o.max_iter == 100 and o.tol <= 1e-12
    assert lib.qp_workspace_bytes(0, 128, 100, 100, 50) >= 128 * (250 * 150 + 100 * 100) * 4
    assert lib.qp_workspace_bytes(0, 0, 100, 100, 50) == 0
    assert lib.qp_workspace_bytes(7, 1, 10, 10, 0) == 0
    assert lib.qp_supported(0, 100, 100, 50) == 0
    assert lib.qp_supported(1, 10, 20, 0) == 0
    assert lib.qp_supported(0, 10, 5, 11) == 1      # more equalities than variables
    assert lib.qp_strerror(0) == b"ok"
    # sizes beyond shared memory run on the global-memory kernel
    assert lib.qp_uses_global_path(0, 100, 100, 50) == 0
    assert lib.qp_uses_global_path(0, 500, 500, 250) == 1
    assert lib.qp_supported(0, 500, 500, 250) == 0
    assert lib.qp_supported(0, 256, 512, 64) == 0
    # the tensor-core setup: FP32 global-path sizes with n + neq ≥ 128 after padding
    assert lib.qp_uses_tensor_cores(None, 0, 500, 500, 250) == 1
    assert lib.qp_uses_tensor_cores(None, 0, 100, 100, 50) == 0     # shared-memory kernel
    assert lib.qp_uses_tensor_cores(None, 1, 500, 500, 250) == 0     # FP64
    assert lib.qp_uses_tensor_cores(None, 0, 64, 512, 16) == 0       # n + neq < 128
    assert lib.qp_uses_tensor_cores(None, 7, 500, 500, 250) == -1
    o = _lib.QPOptions()
    lib.qp_default_options(0, ctypes.byref(o))
    o.path = 1
    assert lib.qp_uses_tensor_cores(ctypes.byref(o), 0, 100, 100, 50) == 1   # forced global
    # the packed plan leaves out the tensor-core panel tiles (its kernels sweep on CUDA cores)
    dims = (ctypes.c_int32 * 3)(500, 500, 250)
    desc = (_lib.QPInstanceDesc * 1)()
    sz = _lib.QPPackedSizes()
    assert lib.qp_packed_plan(None, 0, 1, ctypes.cast(dims, ctypes.c_void_p), desc, ctypes.byref(sz)) == 0
    assert sz.ws_bytes < 256 + lib.qp_workspace_bytes(0, 1, 500, 500, 250)


def test_invalid_arguments_rejected_before_launch():
    lib = _lib.load()
    null = None
    # bad dtype, negative sizes, missing pointers: all return QP_EINVAL without a launch
    assert lib.qp_forward(null, 5, 1, 4, 2, 0, *([null] * 13), 0, null) == 1
    assert lib.qp_forward(null, 0, 1, 0, 2, 0, *([null] * 13), 0, null) == 1
    assert lib.qp_forward(null, 0, 1, 4, 2, 0, *([null] * 13), 0, null) == 1
    assert lib.qp_forward(null, 0, 0, 4, 2, 0, *([null] * 13), 0, null) == 0   # empty batch
    assert lib.qp_backward(null, 0, 1, 4, 2, 0, *([null] * 4), 0, *([null] * 8)) == 1


def test_register_tile_capacity_includes_padding():
    """The shared-memory path is only chosen when the padded sweep matrix fits the register
    tiles (4×4 tiles, at most 4 slots of 512 threads; 2 slots for the Schur complement)."""
    lib = _lib.load()

    def tiles(N):
        nt = (N + 3) // 4
        return nt * (nt + 1) // 2

    for n in range(60, 200, 7):
        for p in range(40, 200, 9):
            for m in (0, 3, 8, n // 4):
                if m > n:
                    continue
                nz = n + (4 - (n + m) % 4) % 4
                fits = tiles(nz + m + p) <= 4 * 512 and tiles(p) <= 2 * 512
                if lib.qp_uses_global_path(0, n, p, m) == 0:
                    assert fits, (n, p, m)


def test_host_copy_many_copies_every_range():
    """qp_host_copy_many (the serving loop's native packing helper; host memory only)."""
    import ctypes
    import numpy as np
    from paper_1703_00443_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(0)
    srcs = [rng.standard_normal(int(k)).astype(np.float32) for k in rng.integers(0, 300000, 37)]
    out = np.zeros(sum(len(a) for a in srcs) + 64, np.float32)
    dst, src, nb, o = [], [], [], 0
    for a in srcs:
        dst.append(out.ctypes.data + 4 * o)
        src.append(a.ctypes.data)
        nb.append(4 * len(a))
        o += len(a)
    k = len(nb)
    for threads in (1, 4):
        out[:] = 0
        rc = lib.qp_host_copy_many(k, (ctypes.c_void_p * k)(*dst), (ctypes.c_void_p * k)(*src),
                                   (ctypes.c_size_t * k)(*nb), threads)
        assert rc == 0
        assert np.array_equal(out[:o], np.concatenate(srcs)) and not out[o:].any()
    assert lib.qp_host_copy_many(-1, None, None, None, 1) != 0
