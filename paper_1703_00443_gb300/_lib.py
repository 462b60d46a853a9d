"""Build and load the in-tree CUDA library ``libqp_gb300.so`` (C ABI of include/qp_gb300.h).

The library is compiled for sm_103a only, in-tree under ``_build/``.  Loading fails loudly
when it is missing: there is no CPU fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libqp_gb300.so")

SOURCES = ["qp_abi", "qp_fwd_f32", "qp_fwd_f64", "qp_bwd", "qp_noalloc", "qp_host", "qp_fwd_variant"]
HEADERS = ["qp_device.cuh", "qp_launch.cuh", "qp_large.cuh", "qp_tc.cuh"]


def _variants():
    """(object name, source, -D flags) of every forward-kernel variant: one object file each,
    so that nvcc compiles them in parallel.  The (SW, CH) pairs match fwd_variant_exists()."""
    out = []
    for T, tag, pairs in (("float", "f32", [(1, 1), (2, 1), (4, 1), (4, 2)]),
                          ("double", "f64", [(1, 1), (2, 1)])):
        out.append((f"fwd_{tag}_large", "qp_fwd_variant", [f"-DQP_T={T}", "-DQP_KIND=1"]))
        for kind, kname in ((0, "plain"), (2, "pksmem"), (3, "pkboth")):
            for sw, ch in pairs:
                out.append((f"fwd_{tag}_{kname}_{sw}{ch}", "qp_fwd_variant",
                            [f"-DQP_T={T}", f"-DQP_KIND={kind}", f"-DQP_SW={sw}", f"-DQP_CH={ch}"]))
    return out


# (object name, source, extra flags); the variants go first, as they take longest
UNITS = _variants() + [(u, u, []) for u in SOURCES if u != "qp_fwd_variant"]

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-Xptxas", "-v"]

_lock = threading.Lock()
_lib = None


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _newest_input() -> float:
    paths = [os.path.join(CSRC, u + ".cu") for u in SOURCES]
    paths += [os.path.join(CSRC, h) for h in HEADERS]
    paths.append(os.path.join(INCLUDE, "qp_gb300.h"))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit (in parallel) and link ``libqp_gb300.so``."""
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    nvcc = _nvcc()

    def compile_unit(unit):
        name, source, defs = unit
        src = os.path.join(CSRC, source + ".cu")
        obj = os.path.join(BUILD, name + ".o")
        log = os.path.join(BUILD, name + ".ptxas.log")
        with open(log, "w") as fh:
            r = subprocess.run([nvcc, *NVCC_FLAGS, *defs, "-c", src, "-o", obj], stdout=fh,
                               stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name} ({source}.cu); see {log}:\n"
                               + open(log).read()[-4000:])
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(len(UNITS), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = LIB + ".tmp"
    r = subprocess.run([nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp,
                        *objs, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


c_int, c_size_t, c_void_p, c_double = ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_double


class QPOptions(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("mu_tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("refine", ctypes.c_int32),
                ("path", ctypes.c_int32), ("time_limit_us", ctypes.c_int32)]


class QPInstanceDesc(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("n", "nineq", "neq", "id", "nz", "flags")] + \
               [(k, ctypes.c_int64) for k in ("oQ", "oq", "oG", "oh", "oA", "ob", "oz", "olam",
                                              "onu", "ows")]


class QPPackedSizes(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("nQ", "nq", "nG", "nh", "nA", "nb", "nz", "nlam",
                                              "nnu", "ws_bytes", "fwd_smem", "bwd_smem")] + \
               [(k, ctypes.c_int32) for k in ("sw", "ch", "n_global", "reserved")]


EXPORTS = {
    "qp_default_options": (None, [c_int, ctypes.POINTER(QPOptions)]),
    "qp_workspace_bytes": (c_size_t, [c_int, c_int, c_int, c_int, c_int]),
    "qp_workspace_bytes_opt": (c_size_t, [ctypes.POINTER(QPOptions), c_int, c_int, c_int, c_int, c_int]),
    "qp_supported": (c_int, [c_int, c_int, c_int, c_int]),
    "qp_uses_global_path": (c_int, [c_int, c_int, c_int, c_int]),
    "qp_uses_tensor_cores": (c_int, [ctypes.POINTER(QPOptions), c_int, c_int, c_int, c_int]),
    "qp_forward": (c_int, [ctypes.POINTER(QPOptions), c_int, c_int, c_int, c_int, c_int]
                   + [c_void_p] * 13 + [c_size_t, c_void_p]),
    "qp_backward": (c_int, [ctypes.POINTER(QPOptions), c_int, c_int, c_int, c_int, c_int]
                    + [c_void_p] * 4 + [c_size_t] + [c_void_p] * 8),
    "qp_backward_ext": (c_int, [ctypes.POINTER(QPOptions), c_int, c_int, c_int, c_int, c_int]
                        + [c_void_p] * 4 + [c_size_t] + [c_void_p] * 11),
    "qp_strerror": (ctypes.c_char_p, [c_int]),
    "qp_host_copy_many": (c_int, [c_int, c_void_p, c_void_p, c_void_p, c_int]),
    "qp_host_pack": (c_int, [c_int, c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p,
                             c_void_p, c_int]),
    "qp_host_unpack": (c_int, [c_int, c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p,
                               c_void_p, c_void_p, c_int]),
    "qp_forward_noalloc": (c_int, [ctypes.POINTER(QPOptions), c_int, c_int, c_int, c_int, c_int]
                           + [c_void_p] * 12 + [c_void_p]),
    "qp_packed_plan": (c_int, [ctypes.POINTER(QPOptions), c_int, c_int, c_void_p,
                               ctypes.POINTER(QPInstanceDesc), ctypes.POINTER(QPPackedSizes)]),
    "qp_packed_plan_ex": (c_int, [ctypes.POINTER(QPOptions), c_int, c_int, c_void_p, c_void_p,
                                  c_void_p, ctypes.POINTER(QPInstanceDesc),
                                  ctypes.POINTER(QPPackedSizes)]),
    "qp_forward_packed": (c_int, [ctypes.POINTER(QPOptions), c_int, c_int, c_void_p,
                                  ctypes.POINTER(QPPackedSizes)] + [c_void_p] * 13 + [c_size_t, c_void_p]),
    "qp_backward_packed": (c_int, [ctypes.POINTER(QPOptions), c_int, c_int, c_void_p,
                                   ctypes.POINTER(QPPackedSizes)] + [c_void_p] * 4 + [c_size_t]
                           + [c_void_p] * 9),
}


def load(path: str | None = None):
    """Load the library (building it first if absent) and declare every exported symbol."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB
        if not os.path.exists(p):
            build()
        lib = ctypes.CDLL(p)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib
