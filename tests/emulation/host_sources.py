"""Host-compilable copies of the library's sources (kernels and host code) for the CPU
checks: the inline PTX and the launch syntax are replaced by host equivalents, everything
else is the library's own code."""
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "..", "..", "paper_1703_00443_gb300", "csrc")


def generate(out):
    os.makedirs(out, exist_ok=True)
    dev = open(os.path.join(SRC, "qp_device.cuh")).read()
    large = open(os.path.join(SRC, "qp_large.cuh")).read()
    dev = dev.replace('#include "qp_large.cuh"', large.replace("#pragma once", ""))
    dev = dev.replace("#include <cuda_runtime.h>", '#define QP_HOST_EMULATION 1\n#include "rt_shim.h"')
    subs = [
        ('asm volatile("prefetch.global.L2 [%0];" :: "l"(c + o));', '(void)(c + o);'),
        ('asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(s), "l"(src) : "memory");',
         '(void)s; std::memcpy(dst_smem, src, 16);'),
        ('asm volatile("cp.async.wait_all;" ::: "memory");', ''),
        ('asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));', 't = emu_time_ns();'),
        ('extern __shared__ __align__(16) unsigned char sm[];', 'unsigned char* sm = emu_dyn_smem;'),
    ]
    for a, b in subs:
        if a not in dev:
            raise RuntimeError("device source changed: " + a)
        dev = dev.replace(a, b)
    if "asm" in re.sub(r"//.*", "", dev):
        raise RuntimeError("inline assembly without a host equivalent")
    dev = re.sub(r"\b__shared__\b", "static", dev)   # one block at a time: statics are per block
    dev = dev.replace("__stcs(", "emu_stcs(")
    open(os.path.join(out, "qp_device.cuh"), "w").write(dev)
    # the tensor-core routines are device-only (under __CUDA_ARCH__); the host build takes
    # the header for its layout functions and runs the CUDA-core sweep
    tc = open(os.path.join(SRC, "qp_tc.cuh")).read()
    tc = re.sub(r"#if defined\(__CUDA_ARCH__\)\n.*?#endif  // __CUDA_ARCH__\n", "", tc, flags=re.S)
    if "asm" in re.sub(r"//.*", "", tc):
        raise RuntimeError("inline assembly left in qp_tc.cuh")
    # the wrappers' host definitions come before the routine that uses them
    tc = tc.replace("// Bounded wait for the completion", '}  // namespace qpk\n#include "tc_emu.h"\n'
                    "namespace qpk {\n// Bounded wait for the completion", 1)
    open(os.path.join(out, "qp_tc.cuh"), "w").write(tc)
    lau = open(os.path.join(SRC, "qp_launch.cuh")).read()
    open(os.path.join(out, "qp_launch.cuh"), "w").write(
        lau.replace("#include <cuda_runtime.h>", '#include "rt_shim.h"'))
    pat = re.compile(r"(\w+)<<<([^,]+),\s*NTHREADS,\s*([^,]+),\s*([^>]+)>>>\((\w+)\);")
    units = []
    for f in ("qp_abi.cu", "qp_fwd_f32.cu", "qp_fwd_f64.cu", "qp_bwd.cu"):
        s = open(os.path.join(SRC, f)).read().replace("#include <cuda_runtime.h>", '#include "rt_shim.h"')
        s = pat.sub(r"emu_launch(\1, \2, \3, \5);", s)
        if "<<<" in s:
            raise RuntimeError("unconverted launch in " + f)
        path = os.path.join(out, f.replace(".cu", ".cpp"))
        open(path, "w").write(s)
        units.append(path)
    # the forward-kernel variants: one host unit per variant, as the library builds them
    var = open(os.path.join(SRC, "qp_fwd_variant.cu")).read().replace(
        "#include <cuda_runtime.h>", '#include "rt_shim.h"')
    var = pat.sub(r"emu_launch(\1, \2, \3, \5);", var)
    if "<<<" in var:
        raise RuntimeError("unconverted launch in qp_fwd_variant.cu")
    for name, _src, defs in variants():
        head = "".join("#define " + d[2:].replace("=", " ", 1) + "\n" for d in defs)
        path = os.path.join(out, name + ".cpp")
        open(path, "w").write(head + var)
        units.append(path)
    return units


def variants():
    """The library's list of forward-kernel variants (read from its build script)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "qp_lib_build", os.path.join(SRC, "..", "_lib.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod._variants()
