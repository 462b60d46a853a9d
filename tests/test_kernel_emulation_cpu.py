"""CPU check of the CUDA kernels' source: the library's kernels and host code, compiled for
the host with shims for the device features they use (one block = 512 host threads with
barriers and per-warp shuffle buffers), run under AddressSanitizer through the C ABI.  Any
access past a buffer (inputs, outputs, workspace, shared memory at its exact launch size)
fails the run, and so does a warp shuffle or barrier that not every thread reaches (it
deadlocks, and the run times out).  The results are checked against the FP64 oracle.  This
is not the product path (that runs only on the GPU); it checks the kernel code for memory
safety and source-level correctness where no GPU is available."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_1703_00443_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
EMU = os.path.join(HERE, "emulation")
BUILD = os.path.join(EMU, "_build")
ROOT = os.path.dirname(HERE)

pytestmark = pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")


@pytest.fixture(scope="module")
def _objects():
    sys.path.insert(0, EMU)
    try:
        import host_sources
    finally:
        sys.path.pop(0)
    units = host_sources.generate(BUILD)
    flags = ["-std=c++20", "-O1", "-g", "-fsanitize=address", "-fno-omit-frame-pointer",
             "-ffp-contract=off", "-I" + BUILD, "-I" + EMU, "-I" + os.path.join(ROOT, "include")]

    def cc(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        r = subprocess.run(["g++", *flags, "-c", src, "-o", obj], capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError(r.stderr[-4000:])
        return obj
    mains = [os.path.join(EMU, "driver.cpp"), os.path.join(EMU, "driver_packed.cpp")]
    with ThreadPoolExecutor(os.cpu_count() or 4) as ex:
        objs = list(ex.map(cc, units + mains))
    return objs[:len(units)], objs[len(units):]


def _link(objs, main, name):
    exe = os.path.join(BUILD, name)
    r = subprocess.run(["g++", "-fsanitize=address", *objs, main, "-o", exe, "-lpthread"],
                       capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError(r.stderr[-4000:])
    return exe


@pytest.fixture(scope="module")
def driver(_objects):
    return _link(_objects[0], _objects[1][0], "driver")


@pytest.fixture(scope="module")
def driver_packed(_objects):
    return _link(_objects[0], _objects[1][1], "driver_packed")


def _run(exe, B, n, p, m, dtype, path, start):
    batch = inputs.random_batch(B, n, p, m, workload=inputs.WL_PLAIN, dtype=dtype, start=start)
    g = inputs.upstream_grad(B, n, workload=inputs.WL_PLAIN, dtype=dtype, start=start)
    tag = f"{B}_{n}_{p}_{m}_{np.dtype(dtype).itemsize}_{path}"
    fin, fout = (os.path.join(BUILD, f"{k}_{tag}.bin") for k in ("in", "out"))
    with open(fin, "wb") as f:
        f.write(np.array([B, n, p, m, 0 if dtype == np.float32 else 1, path], np.int32).tobytes())
        for a in (batch.Q, batch.q, batch.G, batch.h, batch.A, batch.b, g):
            f.write(np.ascontiguousarray(a, dtype=dtype).tobytes())
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0:abort_on_error=1")
    r = subprocess.run([exe, fin, fout], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-4000:]
    o = np.fromfile(fout, dtype=np.uint8)
    es = np.dtype(dtype).itemsize
    counts = [B * n, B * p, B * m, B * n * n, B * n, B * p * n, B * p, B * m * n, B * m]
    vals = np.frombuffer(o[: es * sum(counts)].tobytes(), dtype=dtype).astype(np.float64)
    stat = np.frombuffer(o[es * sum(counts):].tobytes(), dtype=np.int32)
    out, k = [], 0
    for c in counts:
        out.append(vals[k:k + c].reshape(B, -1))
        k += c
    return batch, g, out, stat[:B], stat[B:]


@pytest.mark.parametrize("B,n,p,m,dtype,path,ztol,gtol", [
    (2, 20, 30, 5, np.float32, 0, 1e-5, 1e-4),      # shared-memory path, FP32
    (1, 24, 40, 4, np.float64, 1, 1e-9, 1e-8),      # global-memory path forced, FP64
    (1, 100, 60, 44, np.float32, 1, 1e-5, 1e-4),    # tensor-core setup sweep, 16-pivot last superblock
    (1, 140, 200, 30, np.float32, 0, 1e-5, 1e-4),   # global path by size, two λ tiles
])
def test_emulated_kernels_are_memory_safe_and_match_the_oracle(driver, B, n, p, m, dtype, path,
                                                               ztol, gtol):
    batch, g, out, st, bst = _run(driver, B, n, p, m, dtype, path, start=900)
    # backward status: the forward's code; the near-degenerate flag bit (0x100) may be set
    assert (st == 0).all() and ((bst & 0xFF) == 0).all(), (st, bst)
    names = ("dQ", "dq", "dG", "dh", "dA", "db")
    for i in range(B):
        inst = [np.float64(x) for x in batch.instance(i)]
        sol = oracle.solve(*inst)
        gr = oracle.backward(inst[0], inst[2], inst[3], inst[4], sol, np.float64(g[i]))
        assert np.abs(out[0][i] - sol["z"]).max() <= ztol * max(1.0, np.abs(sol["z"]).max())
        gscale = np.linalg.norm(g[i]) * max(1.0, np.linalg.norm(sol["z"]))
        for a, name in zip(out[3:], names):
            err = np.abs(a[i] - gr[name].reshape(-1)).max() if gr[name].size else 0.0
            assert err <= gtol * max(gscale, np.abs(gr[name]).max(initial=0.0)), (i, name, err)


def test_emulated_packed_batch_both_paths(driver_packed):
    """A packed batch mixing shared-memory-path and global-path instances (sizes whose
    fixed-size setup would take the tensor cores; the packed kernel sweeps on CUDA cores): the
    persistent kernels of both paths and the packed backward, memory-safe and matching the
    oracle."""
    sizes = [(12, 9, 2), (140, 200, 30), (7, 13, 3), (150, 90, 37)]
    inst = [inputs.random_qp(n, p, m, workload=inputs.WL_UNEVEN, index=i, seed=5)
            for i, (n, p, m) in enumerate(sizes)]
    gin = [inputs.upstream_grad(1, n, workload=inputs.WL_UNEVEN, start=i, seed=5)[0]
           for i, (n, p, m) in enumerate(sizes)]
    fin, fout = (os.path.join(BUILD, f"{k}_packed.bin") for k in ("in", "out"))
    with open(fin, "wb") as f:
        f.write(np.array([len(sizes), 0], np.int32).tobytes())
        f.write(np.array(sizes, np.int32).tobytes())
        for t, g in zip(inst, gin):
            for a in tuple(t) + (g,):
                f.write(np.ascontiguousarray(a, dtype=np.float32).tobytes())
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0:abort_on_error=1")
    r = subprocess.run([driver_packed, fin, fout], capture_output=True, text=True, env=env,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    vals = np.fromfile(fout, dtype=np.uint8)
    names = ("z", "lam", "nu", "dQ", "dq", "dG", "dh", "dA", "db")
    k = 0
    res = []
    for (n, p, m) in sizes:
        counts = [n, p, m, n * n, n, p * n, p, m * n, m]
        one = {}
        for name, c in zip(names, counts):
            one[name] = np.frombuffer(vals[k:k + 4 * c].tobytes(), dtype=np.float32).astype(np.float64)
            k += 4 * c
        res.append(one)
    stat = np.frombuffer(vals[k:].tobytes(), dtype=np.int32)
    B = len(sizes)
    assert (stat[:B] == 0).all() and ((stat[B:] & 0xFF) == 0).all(), stat
    for i, (t, g) in enumerate(zip(inst, gin)):
        t = [np.float64(x) for x in t]
        sol = oracle.solve(*t)
        gr = oracle.backward(t[0], t[2], t[3], t[4], sol, np.float64(g))
        assert np.abs(res[i]["z"] - sol["z"]).max() <= 1e-5 * max(1.0, np.abs(sol["z"]).max()), i
        gscale = np.linalg.norm(g) * max(1.0, np.linalg.norm(sol["z"]))
        for name in ("dQ", "dq", "dG", "dh", "dA", "db"):
            ref = gr[name].reshape(-1)
            err = np.abs(res[i][name] - ref).max() if ref.size else 0.0
            assert err <= 1e-4 * max(gscale, np.abs(ref).max(initial=0.0)), (i, name, err)
