"""Serving loop: continuous batching of forward+backward QP requests on one GPU.

Requests (Q, q, G, h, A, b, ∂ℓ/∂z*) of any sizes arrive at any time.  A scheduler thread
admits queued requests, oldest first, into a new packed batch whenever a stream slot is free
and the HBM budget covers the batch (workspace, packed inputs, outputs and gradients).
Requests wait in one queue per size class (by n, thresholds ``size_classes``) and a batch
takes requests of one class, the class whose oldest request is oldest: a batch finishes
with its largest instance, so small requests are not held back by large ones.  Each
admitted batch runs forward and backward (one persistent launch each, ``packed.PackedBatch``)
on its own CUDA stream, so a batch admitted while others are running overlaps with them on
the device; its iterates and factorisation stay in device memory between the two launches.
When a batch's completion event fires, its results are copied to the host, every request's
future is resolved with its own z*, λ*, ν* and gradients, and the batch's slot and budget are
released.  Latency is measured from each request's arrival to the resolution of its future.

Each stream slot keeps one pinned host buffer for a batch's inputs and one for its results,
grown on demand and reused: a batch is packed into sections of the input buffer with numpy
slice copies and moves to the device in one copy, and all its results come back in one copy.
The host copies (requests into the staging buffer, results out of it) go to the library's
native ``qp_host_copy_many`` as one list per batch, which copies on a few host threads
outside the interpreter lock.

Each instance is solved by one thread block on the kernel path its own size selects, so a
request's result does not depend on what it was batched with.
"""
from __future__ import annotations

import collections
import concurrent.futures
import ctypes
import dataclasses
import threading
import time

import numpy as np
import torch

from . import _lib
from .packed import PackedBatch, PackedForward
from .qp import default_options, workspace_bytes

GRAD_KEYS = ("dQ", "dq", "dG", "dh", "dA", "db")


@dataclasses.dataclass
class Request:
    data: tuple                 # (Q, q, G, h, A, b) host arrays
    dl_dz: np.ndarray
    arrival: float              # time.perf_counter() of arrival
    future: concurrent.futures.Future
    nbytes: int = 0
    ptrs: tuple = ()            # host addresses of the six inputs and dl_dz (set by submit)

    @property
    def dims(self):
        Q, _, G, _, A, _ = self.data
        return (Q.shape[0], G.shape[0], A.shape[0])


def request_bytes(dims, dtype=torch.float32) -> int:
    """Device bytes one request holds while in flight: its workspace plus its packed
    inputs, outputs and gradients (offsets padded to 4 elements)."""
    n, p, m = dims
    esz = 4 if dtype == torch.float32 else 8
    r4 = lambda x: (x + 3) // 4 * 4  # noqa: E731
    data = r4(n * n) + r4(n) + r4(p * n) + r4(p) + r4(m * n) + r4(m)
    return workspace_bytes(dtype, 1, n, p, m) + esz * (2 * data + 2 * r4(n) + r4(p) + r4(m)) + 64


class Admission:
    """Admission policy (host logic only): FIFO, a batch takes requests while the HBM budget
    and the batch-size cap allow; a request larger than the whole budget is rejected."""

    def __init__(self, budget_bytes: int, max_batch: int):
        self.budget = int(budget_bytes)
        self.max_batch = int(max_batch)
        self.reserved = 0

    def take(self, queue: collections.deque):
        """Pop the next batch from ``queue``; returns (batch, rejected)."""
        batch, rejected, total = [], [], 0
        while queue and len(batch) < self.max_batch:
            r = queue[0]
            if r.nbytes > self.budget:
                rejected.append(queue.popleft())
                continue
            if self.reserved + total + r.nbytes > self.budget:
                break
            total += r.nbytes
            batch.append(queue.popleft())
        self.reserved += total
        return batch, rejected, total

    def release(self, nbytes: int):
        self.reserved -= int(nbytes)


def _copy_many(dst, src, nbytes, threads):
    """Host copies dst[i] <- src[i] (nbytes[i] bytes; integer addresses) in one native call."""
    k = len(nbytes)
    if k == 0:
        return
    lib = _lib.load()
    rc = lib.qp_host_copy_many(k, (ctypes.c_void_p * k)(*dst), (ctypes.c_void_p * k)(*src),
                               (ctypes.c_size_t * k)(*nbytes), int(threads))
    if rc != 0:
        raise RuntimeError(f"qp_host_copy_many failed: {rc}")


def _sections(sizes, align=64):
    """Offsets of consecutive sections of the given element counts (each at least 1), every
    section starting on a multiple of ``align`` elements; returns (offsets, total)."""
    offs, o = [], 0
    for n in sizes:
        offs.append(o)
        o += (max(int(n), 1) + align - 1) // align * align
    return offs, o


class _Staging:
    """Pinned host buffers of one stream slot, grown on demand (doubling) and reused."""

    def __init__(self, dtype, elems=0):
        self.dtype = dtype
        self.inp = torch.empty(elems, dtype=dtype, pin_memory=elems > 0)
        self.out = torch.empty(elems, dtype=dtype, pin_memory=elems > 0)
        self.status = torch.empty(0, dtype=torch.int32)

    @staticmethod
    def _grow(buf, n, dtype):
        if buf.numel() >= n:
            return buf
        # pinned allocations are slow: leave headroom so steady-state batches reuse the buffer
        return torch.empty(max(n + n // 4, 2 * buf.numel()), dtype=dtype, pin_memory=True)

    def reserve(self, n_in, n_out, n_status):
        self.inp = self._grow(self.inp, n_in, self.dtype)
        self.out = self._grow(self.out, n_out, self.dtype)
        self.status = self._grow(self.status, n_status, torch.int32)


class QPServer:
    def __init__(self, device="cuda:0", dtype=torch.float32, max_inflight=4, max_batch=1024,
                 hbm_budget_bytes=8 << 30, options=None, staging_bytes=16 << 20,
                 copy_threads=None, size_classes=(192,)):
        self.device = torch.device(device)
        self.dtype = dtype
        self.options = options if options is not None else default_options(dtype)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(max_inflight)]
        import os
        self.copy_threads = int(copy_threads or min(8, os.cpu_count() or 1))
        esz = 4 if dtype == torch.float32 else 8
        self.staging = [_Staging(dtype, staging_bytes // esz) for _ in range(max_inflight)]
        self.host_s = {"launch": 0.0, "retire": 0.0}
        self.phase_s = collections.defaultdict(float)   # host time by phase of _launch
        self.free_streams = list(range(max_inflight))
        self.admission = Admission(hbm_budget_bytes, max_batch)
        self.size_classes = tuple(sorted(int(t) for t in size_classes))
        self.queues = [collections.deque() for _ in range(len(self.size_classes) + 1)]
        self.cv = threading.Condition()
        self.inflight = []
        self.max_inflight_seen = 0   # most batches launched and not yet finished at once
        self.latencies = []
        self.batch_sizes = []
        self.completed = 0
        self._stop = False
        self._error = None
        self._thread = threading.Thread(target=self._loop, daemon=True)
        self._thread.start()

    # ------------------------------------------------------------------ client side
    def submit(self, Q, q, G, h, A, b, dl_dz, arrival=None) -> concurrent.futures.Future:
        if self._error is not None:
            raise RuntimeError(f"QP server scheduler failed: {self._error!r}")
        npdt = np.float32 if self.dtype == torch.float32 else np.float64
        data = tuple(np.ascontiguousarray(np.asarray(x), dtype=npdt) for x in (Q, q, G, h, A, b))
        fut = concurrent.futures.Future()
        req = Request(data, np.ascontiguousarray(np.asarray(dl_dz), dtype=npdt),
                      time.perf_counter() if arrival is None else arrival, fut)
        req.nbytes = request_bytes(req.dims, self.dtype)
        req.ptrs = tuple(x.__array_interface__["data"][0] for x in data + (req.dl_dz,))
        with self.cv:
            n = req.dims[0]
            self.queues[sum(n >= t for t in self.size_classes)].append(req)
            self.cv.notify()
        return fut

    def close(self):
        with self.cv:
            self._stop = True
            self.cv.notify()
        self._thread.join()

    def stats(self):
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        nb = max(len(self.batch_sizes), 1)
        return {"completed": self.completed, "batches": len(self.batch_sizes),
                "max_inflight_seen": self.max_inflight_seen,
                "mean_batch": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
                "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "host_launch_ms_per_batch": 1e3 * self.host_s["launch"] / nb,
                "host_retire_ms_per_batch": 1e3 * self.host_s["retire"] / nb,
                "host_launch_phases_ms_per_batch": {k: 1e3 * v / nb for k, v in self.phase_s.items()}}

    # ------------------------------------------------------------------ scheduler
    def _launch(self, reqs, sidx):
        t0 = time.perf_counter()
        stream, stg = self.streams[sidx], self.staging[sidx]
        dims = [r.dims for r in reqs]
        keys = PackedBatch.KEYS
        ph = self.phase_s
        with torch.cuda.stream(stream):
            pb = PackedBatch(dims, dtype=self.dtype, device=self.device, options=self.options)
            t1 = time.perf_counter()
            ph["plan"] += t1 - t0
            tot = pb.totals
            # inputs: Q q G h A b and dℓ/dz; results: z λ ν and the six gradients
            isec, n_in = _sections([tot[k] for k in keys] + [tot["q"]])
            osec, n_out = _sections([tot["q"], tot["h"], tot["b"]] + [tot[k] for k in keys])
            stg.reserve(n_in, n_out, len(reqs))
            # gaps between instances are never read by the kernels
            addr, esz = stg.inp.data_ptr(), stg.inp.element_size()
            dst, src, nbytes = [], [], []
            for j, key in enumerate(keys + ("q",)):
                lens = pb.lengths[key]
                keep = np.nonzero(lens)[0]
                dst += (addr + (isec[j] + pb.offsets[key][keep]) * esz).tolist()
                src += [reqs[i].ptrs[j] for i in keep.tolist()]   # C-contiguous (submit)
                nbytes += (lens[keep] * esz).tolist()
            tc = time.perf_counter()
            ph["pack_lists"] += tc - t1
            _copy_many(dst, src, nbytes, self.copy_threads)
            gbase = isec[len(keys)]
            t2 = time.perf_counter()
            ph["pack_copy"] += t2 - tc
            dev_in = torch.empty(n_in, dtype=self.dtype, device=self.device)
            dev_in.copy_(stg.inp[:n_in], non_blocking=True)
            view = lambda buf, off, n: buf[off:off + max(int(n), 1)]  # noqa: E731
            Q, q, G, h, A, b = (view(dev_in, isec[j], tot[k]) for j, k in enumerate(keys))
            g = view(dev_in, gbase, tot["q"])
            dev_out = torch.zeros(n_out, dtype=self.dtype, device=self.device)
            nB = max(len(reqs), 1)
            fo = PackedForward(view(dev_out, osec[0], tot["q"]), view(dev_out, osec[1], tot["h"]),
                               view(dev_out, osec[2], tot["b"]),
                               torch.empty(nB, dtype=torch.int32, device=self.device),
                               torch.empty(nB, dtype=torch.int32, device=self.device),
                               torch.empty((nB, 4), dtype=torch.float64, device=self.device))
            pb.forward(Q, q, G, h, A, b, out=fo)
            grads = tuple(view(dev_out, osec[3 + j], tot[k]) for j, k in enumerate(keys))
            pb.backward(Q, G, A, g, out=grads)
            stg.out[:n_out].copy_(dev_out, non_blocking=True)
            stg.status[:len(reqs)].copy_(fo.status[:len(reqs)], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        t3 = time.perf_counter()
        ph["device"] += t3 - t2
        self.host_s["launch"] += t3 - t0
        return {"reqs": reqs, "pb": pb, "osec": osec, "n_out": n_out, "event": ev, "stream": sidx,
                "keep": (dev_in, dev_out, fo)}

    def _retire(self, item):
        t0 = time.perf_counter()
        pb, reqs, osec = item["pb"], item["reqs"], item["osec"]
        stg = self.staging[item["stream"]]
        n_out = item["n_out"]
        # one copy out of the staging buffer (in parallel ranges); each request's results view it
        hout = np.empty(n_out, dtype=stg.out.numpy().dtype)
        esz = hout.itemsize
        step = (n_out + self.copy_threads - 1) // self.copy_threads
        starts = range(0, n_out, step)
        _copy_many([hout.ctypes.data + a * esz for a in starts],
                   [stg.out.data_ptr() + a * esz for a in starts],
                   [min(step, n_out - a) * esz for a in starts], self.copy_threads)
        status = stg.status.numpy()
        now = time.perf_counter()
        fields = [("z", "q", osec[0]), ("lam", "h", osec[1]), ("nu", "b", osec[2])] + \
            [(gk, k, osec[3 + j]) for j, (gk, k) in enumerate(zip(GRAD_KEYS, pb.KEYS))]
        for i, r in enumerate(reqs):
            out = {}
            for name, key, base in fields:
                o, l = int(pb.offsets[key][i]), int(pb.lengths[key][i])
                out[name] = hout[base + o:base + o + l].reshape(pb.shapes[key][i])
            out["status"] = int(status[i])
            self.latencies.append(now - r.arrival)
            r.future.set_result(out)
        self.completed += len(reqs)
        self.admission.release(sum(r.nbytes for r in reqs))
        self.free_streams.append(item["stream"])
        self.host_s["retire"] += time.perf_counter() - t0

    def _loop(self):
        try:
            self._schedule()
        except BaseException as exc:   # fail every pending request rather than leave it waiting
            with self.cv:
                pending = [r for q in self.queues for r in q] + \
                    [r for item in self.inflight for r in item["reqs"]]
                for q in self.queues:
                    q.clear()
                self.inflight = []
                self._error = exc
            for r in pending:
                if not r.future.done():
                    r.future.set_exception(RuntimeError(f"QP server scheduler failed: {exc!r}"))
            raise

    def _schedule(self):
        torch.cuda.set_device(self.device)
        while True:
            with self.cv:
                queued = any(self.queues)
                if self._stop and not queued and not self.inflight:
                    return
                if not queued and not self.inflight:
                    self.cv.wait(timeout=0.05)
            progressed = False
            # retire finished batches
            for item in list(self.inflight):
                if item["event"].query():
                    # by identity: items hold arrays, so == between them is not defined
                    self.inflight = [x for x in self.inflight if x is not item]
                    self._retire(item)
                    progressed = True
            # admit new batches while slots and budget allow
            while self.free_streams:
                with self.cv:
                    # the size class whose oldest request is oldest
                    q = min((q for q in self.queues if q), key=lambda q: q[0].arrival, default=None)
                    reqs, rejected, _ = self.admission.take(q) if q is not None else ([], [], 0)
                for r in rejected:
                    r.future.set_exception(MemoryError(
                        f"request needs {r.nbytes} bytes, over the HBM budget {self.admission.budget}"))
                if not reqs:
                    break
                sidx = self.free_streams.pop(0)
                self.inflight.append(self._launch(reqs, sidx))
                self.max_inflight_seen = max(self.max_inflight_seen, len(self.inflight))
                self.batch_sizes.append(len(reqs))
                progressed = True
            if not progressed:
                time.sleep(5e-5)


def poisson_run(server: QPServer, pool, rate: float, count: int, seed: int = 0,
                timeout: float = 600.0):
    """Drive ``server`` with ``count`` requests arriving as a Poisson stream of the given rate
    (requests cycle through ``pool``, a list of (data, dl_dz)).  Returns (results, wall_s)."""
    from .inputs import poisson_arrivals
    arrivals = poisson_arrivals(count, rate, seed=seed)
    futs = []
    t0 = time.perf_counter()
    for k in range(count):
        target = t0 + arrivals[k]
        while True:
            now = time.perf_counter()
            if now >= target:
                break
            # sleep, never spin: a spinning client holds the interpreter lock that the
            # scheduler thread needs (latency still counts from the intended arrival)
            time.sleep(min(target - now, 1e-3))
        data, g = pool[k % len(pool)]
        futs.append(server.submit(*data, g, arrival=target))
    results = [f.result(timeout=timeout) for f in futs]
    return results, time.perf_counter() - t0
