"""Benchmark: batched QP forward+backward solves/s on a GB300.

Workload (one "step"): 128 random dense QPs with n = 100 variables, 100 inequalities and
50 equalities (Q = LLᵀ + 1e-3·I, G, A normal, h = G z0 + s0, b = A z0), FP32 factors with
FP64-accurate residuals, forward (qp_forward) + backward (qp_backward with dℓ/dz* ~ N(0,1)),
all inputs resident in HBM.  L2 is flushed (a 256 MiB write) between timed steps, outside
the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank solves its own batch (instances rank·B .. rank·B+B−1; weak scaling,
no data-path collective); the reported time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

B_DEFAULT, N_DEFAULT, NINEQ_DEFAULT, NEQ_DEFAULT = 128, 100, 100, 50
METRIC = "QP fwd+bwd solves/sec (n=100, batch 128) @ rel err ≤1e-5; p50/p99 latency served"
UNIT = "solves/s"
SM_MAX_MHZ = 2070.0   # GB300 maximum SM clock


def fp32_peak_tflops(sms, mhz=SM_MAX_MHZ):
    """FP32 FMA roofline: SMs × 128 FP32 lanes × 2 flop per FMA × clock."""
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def algorithmic_flops(n, p, m, iters):
    """FLOPs (2 per FMA) of the block-eliminated method per solve: setup factorisations,
    `iters` interior point iterations, the final factorisation and the backward solve."""
    setup = (n ** 3 / 3 + n * n * (p + m) + m * m * n / 2 + m ** 3 / 3 + m * p * n
             + p * p * n / 2 + m * m * p / 2 + p * p * m / 2)
    per_iter = p ** 3 / 3 + 2 * (p * p + 2 * n * p + 2 * n * m + n * n)
    final = p ** 3 / 3 + n * n
    backward = (p * p + 2 * n * p + 2 * n * m + n * n) + n * n + n * p + n * m
    fwd = 2 * (setup + iters * per_iter + final)
    return fwd, 2 * backward


def algorithmic_bytes(n, p, m, esz=4):
    fwd_in = esz * (n * n + n * p + n * m + n + p + m)
    fwd_out = esz * (n + p + m)
    bwd = esz * n + fwd_in
    return fwd_in + fwd_out + bwd


def kernel_source_sha256():
    import glob
    import hashlib
    files = sorted(glob.glob(os.path.join(HERE, "paper_1703_00443_gb300", "csrc", "*.cu")) +
                   glob.glob(os.path.join(HERE, "paper_1703_00443_gb300", "csrc", "*.cuh")))
    h = hashlib.sha256()
    for f in files:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(summary="qp_fwd_kernel_n100_b128.md"):
    """DRAM bytes per launch from the committed ncu summary, or None when the kernel sources
    changed since that capture (the summary records their hash)."""
    path = os.path.join(HERE, "profiles", summary)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.split(":")[0] in ("traffic_bytes_per_launch", "source_sha256"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha256") != kernel_source_sha256():
        return None
    try:
        return int(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def measured_hbm_gbs():
    """The driver's measured copy bandwidth (MEASURED_PEAKS.json), else the recipe's fallback."""
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def bwd_roofline(n, p, m, B, bwd_ms, esz=4):
    """HBM roofline of the backward kernel: algorithmic bytes per solve = ∂ℓ/∂z* in and the six
    gradients out (the workspace the forward left, S/RE and the factor, is read as well and
    reported beside it)."""
    alg = esz * n + esz * (n * n + n * p + n * m + n + p + m)
    m1 = n + (4 - (n + m) % 4) % 4 + m   # n padded to make n + neq a multiple of 4, plus neq
    ws_read = esz * ((m1 + p) * m1 + p * p)
    peak, src = measured_hbm_gbs()
    achieved = alg * B / (bwd_ms / 1e3) / 1e9
    return {"bound": "hbm", "kernel": "qp_bwd_kernel", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "peak_source": src + " copy bandwidth",
            "algorithmic_bytes_per_launch": alg * B, "workspace_bytes_read_per_launch": ws_read * B,
            "traffic": profiled_traffic("qp_bwd_kernel_n100_b128.md")}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples (the JSON line carries their summary); BENCH_CLOCKS_DIR keeps them
        import tempfile
        self.path = os.path.join(os.environ.get("BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"qp_bench_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index),
                                          f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


# ----------------------------------------------------------------------------- oracle legs
RESULTS = ("z", "lam", "nu", "dQ", "dq", "dG", "dh", "dA", "db")


def _oracle_instance(args):
    """Forward + backward of one instance with the FP64 oracle (runs in a worker process);
    returns its index, the time taken and every result."""
    n, p, m, idx = args
    import oracle
    from paper_1703_00443_gb300 import inputs
    Q, q, G, h, A, b = inputs.random_qp(n, p, m, workload=inputs.WL_SWEEP, index=idx,
                                        dtype=np.float32)
    g = inputs.upstream_grad(1, n, workload=inputs.WL_SWEEP, start=idx)[0].astype(np.float64)
    t0 = time.perf_counter()
    sol = oracle.solve(Q, q, G, h, A, b)
    gr = oracle.backward(Q, G, h, A, sol, g)
    dt = time.perf_counter() - t0
    res = {k: sol[k] for k in ("z", "lam", "nu")}
    res.update({k: gr[k] for k in ("dQ", "dq", "dG", "dh", "dA", "db")})
    return idx, dt, res, g


def _oracle_pool(workers):
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                            "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    pool = mp.get_context("spawn").Pool(workers)
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    return pool


def accuracy_vs_oracle(gpu_out, done):
    """Worst error of every GPU result against the FP64 oracle over the given instances, in
    the two forms of the relative error: ‖x − x_ref‖₂/max(‖x_ref‖₂, floor) and
    max_i |x_i − x_ref,i|/max(‖x_ref‖∞, floor).  floor = 1e-12 for z*, λ*, ν*; for a
    gradient 1e-3·‖∂ℓ/∂z*‖ (times max(1, ‖z*‖) for dQ, dG, dA), because a gradient can vanish
    identically at the solution (e.g. dq at a vertex)."""
    worst = {}
    for idx, _, ref, g in done:
        for k in RESULTS:
            r = np.asarray(ref[k], dtype=np.float64).ravel()
            x = np.asarray(gpu_out[k][idx], dtype=np.float64).ravel()
            if r.size == 0:
                continue
            for form, ordv in (("l2", None), ("inf", np.inf)):
                fl = 1e-12
                if k.startswith("d"):
                    fl = 1e-3 * np.linalg.norm(g, ord=ordv)
                    if k in ("dQ", "dG", "dA"):
                        fl *= max(1.0, np.linalg.norm(ref["z"], ord=ordv))
                e = np.linalg.norm(x - r, ord=ordv) / max(np.linalg.norm(r, ord=ordv), fl)
                key = f"{k}_{form}"
                worst[key] = max(worst.get(key, 0.0), float(e))
    return {"instances": len(done), "rel_err_max": worst,
            "bar": {"z": 1e-5, "gradients": 1e-4, "lam_nu": 1e-4},
            "within_bar": all(v <= (1e-5 if k.startswith("z_") else 1e-4)
                              for k, v in worst.items())}


def cpu_baseline(n, p, m, budget_s=15.0, gpu_out=None):
    """The oracle as it stands, one instance per process (BLAS threads = 1), all host cores,
    on a bounded sample of the same instances (timed), and on one core; then, untimed, the
    rest of the batch so that every GPU result of the step is checked against FP64."""
    cores = os.cpu_count() or 1
    pool = _oracle_pool(cores)
    try:
        pool.map(_oracle_instance, [(n, p, m, 0)] * cores)   # warm up the workers
        t0 = time.perf_counter()
        done = []
        batch_idx = 0
        while time.perf_counter() - t0 < budget_s and batch_idx * cores < B_DEFAULT:
            idxs = [batch_idx * cores + k for k in range(cores)]
            done += pool.map(_oracle_instance, [(n, p, m, i) for i in idxs if i < B_DEFAULT])
            batch_idx += 1
        wall = time.perf_counter() - t0
        timed = len(done)
        if gpu_out is not None:
            have = {d[0] for d in done}
            done += pool.map(_oracle_instance, [(n, p, m, i) for i in range(B_DEFAULT)
                                                if i not in have])
    finally:
        pool.close()
        pool.join()
    # one core, in this process: a few instances
    t1 = time.perf_counter()
    k1 = 0
    while k1 < 8 and (k1 == 0 or time.perf_counter() - t1 < budget_s / 3):
        _oracle_instance((n, p, m, k1))
        k1 += 1
    one = k1 / (time.perf_counter() - t1)
    res = {"value": timed / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{timed} of the {B_DEFAULT} step instances (n={n}, nineq={p}, neq={m}), "
                     f"FP64 dense-KKT PDIPM fwd+bwd, one instance per process, BLAS threads 1",
           "one_core": {"value": one, "unit": UNIT, "cores": 1,
                        "sample": f"{k1} instances in one process"}}
    acc = accuracy_vs_oracle(gpu_out, done) if gpu_out is not None and done else None
    return res, acc


def _classes(args):
    return tuple(int(v) for v in str(args.serve_classes).split(",") if v)


def serving_run(dev, rates, count, inflight=4, classes=(192,), max_batch=512):
    """Poisson streams of fwd+bwd requests (n log-uniform in [16, 512], nineq = n, neq = n/4)
    through the continuous-batching server, one run per offered rate; p50/p99 latency from
    arrival to result, throughput, and the scheduler's host time per batch."""
    from paper_1703_00443_gb300 import inputs
    from paper_1703_00443_gb300.serving import QPServer, poisson_run
    sizes = inputs.serve_sizes(128)
    pool = []
    for i, (nn, pp, mm) in enumerate(sizes):
        data = inputs.random_qp(nn, pp, mm, workload=inputs.WL_SERVE, index=i)
        gg = inputs.upstream_grad(1, nn, workload=inputs.WL_SERVE, start=i)[0]
        pool.append((tuple(np.float32(x) for x in data), np.float32(gg)))
    server = QPServer(device=dev, max_inflight=inflight, max_batch=max_batch,
                      size_classes=tuple(classes))
    runs = []
    try:
        # warm-up at the highest offered rate, so batches reach their steady-state sizes and
        # the server's pinned staging buffers their final size before anything is timed
        poisson_run(server, pool, max(rates), min(1000, count), seed=99)
        server.equalize_staging()   # every slot sized for the largest batch seen
        for k, rate in enumerate(rates):
            server.latencies.clear()
            server.batch_sizes.clear()
            server.completed = 0
            server.host_s = {"launch": 0.0, "retire": 0.0}
            server.phase_s.clear()
            results, wall = poisson_run(server, pool, rate, count, seed=1 + k)
            st = server.stats()
            bad = sum(r["status"] != 0 for r in results)
            runs.append({"rate_req_s": rate, "requests": count, "throughput_req_s": count / wall,
                         "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "batches": st["batches"],
                         "mean_batch": st["mean_batch"], "nonconverged": int(bad),
                         "host_ms_per_batch": st["host_launch_ms_per_batch"] +
                         st["host_retire_ms_per_batch"],
                         "host_ms_by_phase": dict(st["host_launch_phases_ms_per_batch"],
                                                  retire=st["host_retire_ms_per_batch"])})
    finally:
        server.close()
    return {"runs": runs, "max_inflight": inflight, "size_classes": list(classes),
            "max_batch": max_batch, "requests_per_rate": count,
            "batched_same_mix": batched_same_mix(dev, pool, 512),
            "workload": "n log-uniform [16,512], nineq=n, neq=n/4, fwd+bwd, host arrays in/out"}


def batched_same_mix(dev, pool, count, steps=3):
    """The plain batched path on the serving stream's request mix: `count` requests (the pool
    cycled) known up front, solved as one packed batch with inputs resident on the device;
    fwd+bwd requests per second, the ceiling the served rates are compared with."""
    import torch
    from paper_1703_00443_gb300.packed import PackedBatch
    reqs = [pool[k % len(pool)] for k in range(count)]
    sizes = [(d[0].shape[0], d[2].shape[0], d[4].shape[0]) for d, _ in reqs]
    pb = PackedBatch(sizes, device=dev)
    P = pb.pack([d for d, _ in reqs])
    G1 = pb.pack_vec([g for _, g in reqs], "q")
    fo = pb.forward(*P)
    go = pb.backward(P[0], P[2], P[4], G1)
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pb.forward(*P, out=fo)
        pb.backward(P[0], P[2], P[4], G1, out=go)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    tm = statistics.mean(ms)
    return {"requests": count, "ms": tm, "throughput_req_s": count / (tm / 1e3),
            "note": "one packed batch, inputs resident on the device, no host copies"}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    n, p, m = N_DEFAULT, NINEQ_DEFAULT, NEQ_DEFAULT
    cores = os.cpu_count() or 1
    pool = _oracle_pool(cores)
    per_step = cores   # each step: one instance per core (a bounded sample of the batch)
    try:
        for w in range(args.warmup):
            pool.map(_oracle_instance, [(n, p, m, k) for k in range(per_step)])
        times = []
        for s in range(args.steps):
            t0 = time.perf_counter()
            pool.map(_oracle_instance, [(n, p, m, (s * per_step + k) % B_DEFAULT)
                                        for k in range(per_step)])
            times.append(time.perf_counter() - t0)
    finally:
        pool.close()
        pool.join()
    tot = sum(times)
    value = per_step * args.steps / tot
    # n_gpus: the launch this line belongs to (the oracle itself runs on rank 0's host cores)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"random dense QP fwd+bwd, n={n}, nineq={p}, neq={m}, batch {B_DEFAULT}",
                       "n": n, "nineq": p, "neq": m, "batch": B_DEFAULT,
                       "step": f"{per_step} instances of the batch per step (bounded sample)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} instances per step, one per process, BLAS threads 1"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def rank_batch(rank, B, n, p, m):
    """The batch rank `rank` solves: instances rank·B … rank·B+B−1 of the benchmark's seeded
    stream, so ranks work on disjoint instances (weak scaling) and the union over N ranks is
    the single-process batch of N·B instances."""
    from paper_1703_00443_gb300 import inputs
    batch = inputs.random_batch(B, n, p, m, workload=inputs.WL_SWEEP, dtype=np.float32,
                                start=rank * B)
    g = inputs.upstream_grad(B, n, workload=inputs.WL_SWEEP, start=rank * B)
    return batch, g


def max_over_ranks(values, device, dist=None):
    """Element-wise maximum of per-rank timings across the process group (or the values
    themselves when there is no group)."""
    import torch
    t = torch.tensor(values, device=device, dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_rate(world, per_rank_batch, ms):
    """Solves per second of the whole job: all ranks' instances over the slowest rank's time."""
    return world * per_rank_batch / (ms / 1e3)


def run_gpu(args):
    import torch

    from paper_1703_00443_gb300 import qp_backward, qp_forward
    from paper_1703_00443_gb300.qp import alloc_workspace

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B, n, p, m = args.batch, N_DEFAULT, NINEQ_DEFAULT, NEQ_DEFAULT
    batch, g = rank_batch(rank, B, n, p, m)
    host = [batch.Q, batch.q, batch.G, batch.h, batch.A, batch.b, g]
    dev_in = [torch.from_numpy(x).to(dev) for x in host]
    Q, q, G, h, A, b, dl = dev_in
    wsbuf = alloc_workspace(torch.float32, B, n, p, m, dev)
    z = torch.empty((B, n), device=dev)
    lam = torch.empty((B, p), device=dev)
    nu = torch.empty((B, m), device=dev)
    st = torch.empty((B,), device=dev, dtype=torch.int32)
    it = torch.empty((B,), device=dev, dtype=torch.int32)
    gout = [torch.empty(s, device=dev) for s in [(B, n, n), (B, n), (B, p, n), (B, p), (B, m, n), (B, m)]]
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        fwd = qp_forward(Q, q, G, h, A, b, workspace=wsbuf, out=(z, lam, nu, st, it))
        qp_backward(fwd, dl, out=gout)
        return fwd

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        e0, e1, e2 = ev[k]
        e0.record(stream)
        fwd = qp_forward(Q, q, G, h, A, b, workspace=wsbuf, out=(z, lam, nu, st, it))
        e1.record(stream)
        qp_backward(fwd, dl, out=gout)
        e2.record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    fwd_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)]
    bwd_ms = [ev[k][1].elapsed_time(ev[k][2]) for k in range(args.steps)]
    step_ms = sum(fwd_ms) / args.steps + sum(bwd_ms) / args.steps

    # End to end through the public API: pinned host inputs -> device, solve, read back
    # z* and the six gradients each step.
    pinned = [torch.from_numpy(x).pin_memory() for x in host]
    outs_h = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in [z] + gout]
    h2d = sum(t.numel() * t.element_size() for t in pinned)
    d2h = sum(t.numel() * t.element_size() for t in outs_h)
    e2e_ms = []
    for k in range(args.steps + 2):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for d, hsrc in zip(dev_in, pinned):
            d.copy_(hsrc, non_blocking=True)
        fwd = qp_forward(Q, q, G, h, A, b, workspace=wsbuf, out=(z, lam, nu, st, it))
        qp_backward(fwd, dl, out=gout)
        for hdst, d in zip(outs_h, [z] + gout):
            hdst.copy_(d, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if k >= 2:
            e2e_ms.append(e0.elapsed_time(e1))
    clocks = sampler.stop()

    # The same 128 instances through the packed (persistent, uneven-capable) path.
    packed_ms = None
    if not args.no_extras:
        from paper_1703_00443_gb300.packed import PackedBatch
        pb = PackedBatch([(n, p, m)] * B, device=dev)
        Pq = [pb.pack_vec([x[i] for i in range(B)], k) for x, k in
              zip((batch.Q, batch.q, batch.G, batch.h, batch.A, batch.b), pb.KEYS)]
        Pg = pb.pack_vec([g[i] for i in range(B)], "q")
        fo = pb.forward(*Pq)
        go = pb.backward(Pq[0], Pq[2], Pq[4], Pg)
        torch.cuda.synchronize()
        pms = []
        for k in range(max(10, args.steps // 5)):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pb.forward(*Pq, out=fo)
            pb.backward(Pq[0], Pq[2], Pq[4], Pg, out=go)
            e1.record(stream)
            e1.synchronize()
            pms.append(e0.elapsed_time(e1))
        packed_ms = statistics.mean(pms)

    # Max over ranks.
    step_ms, fwd_mean, e2e_mean = max_over_ranks(
        [step_ms, sum(fwd_ms) / args.steps, statistics.mean(e2e_ms)], dev,
        dist if ws > 1 else None)
    status = st.cpu().numpy()
    iters = it.cpu().numpy()
    if rank != 0:
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    value = whole_job_rate(ws, B, step_ms)
    e2e_value = whole_job_rate(ws, B, e2e_mean)
    k_mean = float(iters.mean())
    f_fwd, f_bwd = algorithmic_flops(n, p, m, k_mean)
    achieved = f_fwd * B / (fwd_mean / 1e3) / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = fp32_peak_tflops(sms)
    gpu_out = {"z": z.cpu().numpy(), "lam": lam.cpu().numpy(), "nu": nu.cpu().numpy()}
    gpu_out.update({k: t.cpu().numpy() for k, t in zip(("dQ", "dq", "dG", "dh", "dA", "db"), gout)})
    # backward status words of the step (flag bits mark nearly degenerate solutions)
    bstat = torch.empty((B,), device=dev, dtype=torch.int32)
    qp_backward(fwd, dl, out=[torch.empty_like(t) for t in gout], status=bstat)
    bstat = bstat.cpu().numpy()
    uneven = None
    if not args.no_extras and ws == 1:
        uneven = {"untuned": uneven_run(dev, args.uneven_count, args.uneven_steps, False, flush, stream)}
        if not args.no_tune:
            uneven["tuned"] = uneven_run(dev, args.uneven_count, args.uneven_steps, True, flush, stream)
    served = None
    if not args.no_extras and ws == 1:
        served = serving_run(dev, [float(r) for r in str(args.serve_rate).split(",")],
                             args.serve_count, args.serve_inflight, _classes(args),
                             args.serve_max_batch)
    cpu, acc = (None, None)
    if not args.no_cpu_baseline and ws == 1:
        cpu, acc = cpu_baseline(n, p, m, budget_s=args.cpu_budget, gpu_out=gpu_out)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded random QPs, recipe of the paper's timing experiment)",
        "config": {"workload": f"random dense QP fwd+bwd, n={n}, nineq={p}, neq={m}, batch {B}",
                   "n": n, "nineq": p, "neq": m, "batch": B, "per_gpu_batch": B,
                   "precision": "FP32 factors, FP64-accurate residual/iterate/refinement",
                   "l2": "flushed between timed steps (256 MiB write, outside the events)",
                   "parallelism": f"independent batches per GPU x{ws}",
                   "fwd_ms": fwd_mean, "bwd_ms": step_ms - fwd_mean,
                   "iters_mean": k_mean, "iters_max": int(iters.max()),
                   "status_counts": {str(s): int((status == s).sum()) for s in np.unique(status)},
                   "near_degenerate": int(((bstat & 0x100) != 0).sum()),
                   "wall_s_timed_loop": t_wall},
        "roofline": {"bound": "alu", "kernel": "qp_fwd_kernel", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_source": f"{sms} SMs (device properties) x 128 FP32 lanes x 2 x "
                                    f"{SM_MAX_MHZ:.0f} MHz (nominal; MEASURED_PEAKS.json has no "
                                    "FP32 figure)",
                     "traffic": profiled_traffic(),
                     "traffic_unit": "bytes per launch (dram read+write, ncu)",
                     "algorithmic_flops_per_launch": f_fwd * B},
        "roofline_bwd": bwd_roofline(n, p, m, B, step_ms - fwd_mean),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 2 * args.steps,
        "batched_vs_plain": None if packed_ms is None else {
            "plain_fixed_size_ms_per_step": step_ms, "packed_persistent_ms_per_step": packed_ms,
            "note": "same 128 instances; packed = one persistent launch per direction over descriptors"},
        "uneven": uneven,
        "served": served,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "accuracy_vs_oracle": acc,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def _time_fixed(Tin, gdev, steps, flush, stream):
    """Mean device time (ms) of one fwd+bwd step of the fixed-size path (L2 flushed)."""
    import torch
    from paper_1703_00443_gb300 import qp_backward, qp_forward
    f = qp_forward(*Tin)
    go = qp_backward(f, gdev)
    for _ in range(2):
        f = qp_forward(*Tin, workspace=f.workspace, out=(f.z, f.lam, f.nu, f.status, f.iters, f.resid))
        qp_backward(f, gdev, out=go)
    torch.cuda.synchronize()
    ms = []
    for k in range(steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f = qp_forward(*Tin, workspace=f.workspace, out=(f.z, f.lam, f.nu, f.status, f.iters, f.resid))
        qp_backward(f, gdev, out=go)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.mean(ms), f


def uneven_run(dev, count, steps, tuned, flush, stream):
    """The uneven workload: `count` QPs with n ~ U{8..256}, nineq ~ U{n/2..2n}, neq ~ U{0..n/4}
    as one packed batch, forward (global-path and shared-memory-path instances in two
    persistent kernels side by side) + backward (one persistent kernel), L2 flushed between
    steps.  tuned: the autotuner's path choice and cost model."""
    import torch
    from paper_1703_00443_gb300 import inputs
    from paper_1703_00443_gb300.packed import PackedBatch
    sizes = inputs.uneven_sizes(count)
    tuning = None
    t0 = time.perf_counter()
    if tuned:
        from paper_1703_00443_gb300 import autotune
        tuning = autotune.autotune(device=dev, save_to=None)
    pb = PackedBatch(sizes, device=dev, tuning=tuning)
    inst = [inputs.random_qp(nn, pp, mm, workload=inputs.WL_UNEVEN, index=i)
            for i, (nn, pp, mm) in enumerate(sizes)]
    gl = [inputs.upstream_grad(1, nn, workload=inputs.WL_UNEVEN, start=i)[0]
          for i, (nn, pp, mm) in enumerate(sizes)]
    P = pb.pack([tuple(np.float32(x) for x in t) for t in inst])
    G1 = pb.pack_vec([np.float32(x) for x in gl], "q")
    tune_s = time.perf_counter() - t0
    fo = pb.forward(*P)
    go = pb.backward(P[0], P[2], P[4], G1)
    torch.cuda.synchronize()
    ms = []
    for k in range(steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pb.forward(*P, out=fo)
        pb.backward(P[0], P[2], P[4], G1, out=go)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    tm = statistics.mean(ms)
    st = fo.status[:count].cpu().numpy()
    return {"value": count / (tm / 1e3), "unit": UNIT, "ms_per_step": tm, "steps": steps,
            "count": count, "global_path_instances": pb.n_global,
            "tuned": bool(tuned), "tuning_s": tune_s if tuned else 0.0,
            "workspace_gb": int(pb.sizes.ws_bytes) / 1e9,
            "iters_mean": float(fo.iters[:count].float().mean()),
            "converged": int((st == 0).sum()),
            "sizes": "n~U{8..256}, nineq~U{n/2..2n}, neq~U{0..n/4}"}


def run_workload(args):
    """Secondary workloads, one JSON line each (not the headline metric)."""
    import torch
    from paper_1703_00443_gb300 import inputs
    from paper_1703_00443_gb300.packed import PackedBatch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)
    stream = torch.cuda.current_stream(dev)
    line = {"workload": args.workload, "unit": UNIT, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "l2": "flushed between timed steps"}
    if args.workload == "sweep":
        rows = []
        grid = [(n, B) for n in (10, 50, 100, 500) for B in (1, 64, 128)]
        if args.sweep_sizes:   # e.g. "500:1" for a one-launch profiling case
            grid = [tuple(int(v) for v in item.split(":")) for item in args.sweep_sizes.split(",")]
        for n, B in grid:
            p, m = n, n // 2
            bt = inputs.random_batch(B, n, p, m, workload=inputs.WL_SWEEP)
            g = inputs.upstream_grad(B, n, workload=inputs.WL_SWEEP)
            Tin = [torch.from_numpy(x).to(dev) for x in (bt.Q, bt.q, bt.G, bt.h, bt.A, bt.b)]
            steps = 5 if n == 500 else 20
            ms, f = _time_fixed(Tin, torch.from_numpy(g).to(dev), steps, flush, stream)
            rows.append({"n": n, "nineq": p, "neq": m, "batch": B, "ms_per_step": ms,
                         "solves_per_s": B / (ms / 1e3),
                         "iters_mean": float(f.iters.float().mean()),
                         "converged": int((f.status == 0).sum())})
        line.update({"metric": "QP fwd+bwd solves/sec, timing sweep (n, nineq=n, neq=n/2)",
                     "sweep": rows})
    elif args.workload == "onehot":
        B, n, m = 512, 64, 40
        bt = inputs.onehot_batch(B, n, m)
        tgt = torch.from_numpy(inputs.onehot_target(B, n)).to(dev)
        Tin = [torch.from_numpy(x).to(dev) for x in (bt.Q, bt.q, bt.G, bt.h, bt.A, bt.b)]
        from paper_1703_00443_gb300 import qp_forward
        z = qp_forward(*Tin).z
        gdev = (2.0 / n) * (z - tgt)
        ms, f = _time_fixed(Tin, gdev, 20, flush, stream)
        line.update({"metric": "structured one-hot QP fwd+bwd solves/sec (n=64, neq=40, z>=0, batch 512)",
                     "value": B / (ms / 1e3), "ms_per_step": ms,
                     "iters_mean": float(f.iters.float().mean()), "converged": int((f.status == 0).sum())})
    elif args.workload == "serving":
        line.update({"metric": "served fwd+bwd requests/sec and p50/p99 latency (Poisson arrivals)",
                     "unit": "req/s"})
        line.update(serving_run(dev, [float(r) for r in str(args.serve_rate).split(",")],
                                args.serve_count, args.serve_inflight, _classes(args),
                                args.serve_max_batch))
    elif args.workload == "uneven":
        line.update({"metric": "uneven batch fwd+bwd solves/sec (two persistent kernels forward, one backward)"})
        line.update(uneven_run(dev, args.uneven_count, args.uneven_steps, args.tuned, flush, stream))
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", type=int, default=B_DEFAULT)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-extras", action="store_true", help="skip the packed and serving runs")
    ap.add_argument("--serve-rate", default="1000,3000,10000,30000,100000",
                    help="offered request rates (req/s), comma-separated")
    ap.add_argument("--serve-count", type=int, default=5000)
    ap.add_argument("--serve-inflight", type=int, default=16, help="server stream slots")
    ap.add_argument("--serve-classes", default="64,160,320", help="size-class thresholds on n")
    ap.add_argument("--serve-max-batch", type=int, default=256)
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "sweep", "onehot", "uneven", "serving"])
    ap.add_argument("--uneven-count", type=int, default=4096)
    ap.add_argument("--sweep-sizes", default="",
                    help="sweep points n:batch, comma-separated (default: the full grid)")
    ap.add_argument("--uneven-steps", type=int, default=3)
    ap.add_argument("--tuned", action="store_true", help="autotune the packed schedule first")
    ap.add_argument("--no-tune", action="store_true",
                    help="main line: report the uneven workload untuned only")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "headline":
        run_workload(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
