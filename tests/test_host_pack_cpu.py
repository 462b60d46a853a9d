"""The serving loop's native gather/scatter (qp_host_pack / qp_host_unpack) against numpy,
on a packed plan made on the host (no GPU involved)."""
import ctypes

import numpy as np
import pytest

from paper_1703_00443_gb300 import _lib, inputs
from paper_1703_00443_gb300.serving import (FIELDS_IN, FIELDS_OUT, OUT_NAMES, ServedResult,
                                            _sections)

RULES = {0: ("oQ", lambda n, p, m: n * n), 1: ("oq", lambda n, p, m: n),
         2: ("oG", lambda n, p, m: p * n), 3: ("oh", lambda n, p, m: p),
         4: ("oA", lambda n, p, m: m * n), 5: ("ob", lambda n, p, m: m)}


def _plan(sizes, code=0):
    lib = _lib.load()
    B = len(sizes)
    dims = np.ascontiguousarray(np.array(sizes, dtype=np.int32).reshape(-1, 3))
    desc = (_lib.QPInstanceDesc * B)()
    s = _lib.QPPackedSizes()
    o = _lib.QPOptions()
    lib.qp_default_options(code, ctypes.byref(o))
    assert lib.qp_packed_plan_ex(ctypes.byref(o), code, B, dims.ctypes.data_as(ctypes.c_void_p),
                                 None, None, desc, ctypes.byref(s)) == 0
    return desc, s


def _totals(s, fields):
    key = {0: "nQ", 1: "nq", 2: "nG", 3: "nh", 4: "nA", 5: "nb"}
    return [getattr(s, key[f]) for f in fields]


@pytest.mark.parametrize("dtype,code", [(np.float32, 0), (np.float64, 1)])
def test_pack_places_every_array_at_its_planned_offset(dtype, code):
    sizes = inputs.uneven_sizes(37, seed=3) + [(5, 0, 0), (9, 4, 0), (6, 0, 2)]
    desc, s = _plan(sizes, code)
    B = len(sizes)
    rng = np.random.default_rng(0)
    arrs = [[rng.standard_normal(RULES[f][1](*sizes[i])).astype(dtype) for f in FIELDS_IN]
            for i in range(B)]
    sec, total = _sections(_totals(s, FIELDS_IN))
    buf = np.full(total, np.nan, dtype=dtype)
    src = (ctypes.c_void_p * (7 * B))(*[a.ctypes.data for row in arrs for a in row])
    lib = _lib.load()
    assert lib.qp_host_pack(B, desc, buf.itemsize, 7, (ctypes.c_int32 * 7)(*FIELDS_IN),
                            (ctypes.c_int64 * 7)(*sec), src, buf.ctypes.data, 4) == 0
    for k in range(B):
        d = desc[k]
        for f, (rule, a) in enumerate(zip(FIELDS_IN, arrs[d.id])):
            o = sec[f] + getattr(d, RULES[rule][0])
            assert np.array_equal(buf[o:o + a.size], a), (d.id, f)


@pytest.mark.parametrize("threads", [1, 8])
def test_unpack_gathers_each_instance_contiguously(threads):
    sizes = [(n, 2 * n, n // 4) for n in (3, 40, 7, 120, 64)] * 30   # > 1 MiB: threaded
    desc, s = _plan(sizes)
    B = len(sizes)
    sec, total = _sections(_totals(s, FIELDS_OUT))
    src = np.arange(total, dtype=np.float32)
    dst = np.full(sum(sum(RULES[f][1](*sz) for f in FIELDS_OUT) for sz in sizes), -1.0,
                  dtype=np.float32)
    off = np.empty(B + 1, dtype=np.int64)
    lib = _lib.load()
    assert lib.qp_host_unpack(B, desc, 4, 9, (ctypes.c_int32 * 9)(*FIELDS_OUT),
                              (ctypes.c_int64 * 9)(*sec), src.ctypes.data, dst.ctypes.data,
                              off.ctypes.data, threads) == 0
    assert off[B] == dst.size and (dst >= 0).all()
    by_id = {desc[k].id: desc[k] for k in range(B)}
    for i in range(B):
        d = by_id[i]
        res = ServedResult(dst, off[i], sizes[i], 0)
        for f, (rule, name) in enumerate(zip(FIELDS_OUT, OUT_NAMES)):
            o = sec[f] + getattr(d, RULES[rule][0])
            want = src[o:o + RULES[rule][1](*sizes[i])]
            assert np.array_equal(res[name].reshape(-1), want), (i, name)
        assert res["z"].shape == (sizes[i][0],) and res["dG"].shape == (sizes[i][1], sizes[i][0])
        assert set(res) == set(OUT_NAMES) | {"status"} and res["status"] == 0


def test_pack_rejects_bad_arguments():
    desc, s = _plan([(4, 2, 1)])
    lib = _lib.load()
    f = (ctypes.c_int32 * 1)(17)
    sec = (ctypes.c_int64 * 1)(0)
    buf = np.zeros(64, dtype=np.float32)
    src = (ctypes.c_void_p * 1)(buf.ctypes.data)
    assert lib.qp_host_pack(1, desc, 4, 1, f, sec, src, buf.ctypes.data, 1) == 1   # bad rule
    assert lib.qp_host_pack(1, desc, 3, 1, (ctypes.c_int32 * 1)(0), sec, src, buf.ctypes.data, 1) == 1
    assert lib.qp_host_pack(0, None, 4, 1, f, sec, src, buf.ctypes.data, 1) == 0
