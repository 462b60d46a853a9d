"""Serving loop: continuous batching of forward+backward QP requests on one GPU.

Requests (Q, q, G, h, A, b, ∂ℓ/∂z*) of any sizes arrive at any time.  A scheduler thread
admits queued requests, oldest first, into a new packed batch whenever a stream slot is free
and the HBM budget covers the batch (workspace, packed inputs, outputs and gradients).
Requests wait in one queue per size class (by n, thresholds ``size_classes``) and a batch
takes requests of one class, the class whose oldest request is oldest: a batch finishes
with its largest instance, so small requests are not held back by large ones.  Each
admitted batch runs forward and backward (``qp_forward_packed`` / ``qp_backward_packed``)
on its own CUDA stream, so a batch admitted while others are running overlaps with them on
the device; its iterates and factorisation stay in device memory between the two launches.
When a batch's completion event fires, its results are copied to the host, every request's
future is resolved with its own z*, λ*, ν* and gradients, and the batch's slot and budget are
released.  Latency is measured from each request's arrival to the resolution of its future.

Each stream slot keeps one pinned host buffer for a batch's inputs and one for its results,
grown on demand and reused.  The per-batch host work runs in native calls that release the
interpreter lock: ``qp_packed_plan_ex`` plans the batch, ``qp_host_pack`` gathers every
request's arrays (and the descriptors) into the input buffer, which moves to the device in
one copy; the results come back in one copy and ``qp_host_unpack`` scatters them into one
host array per batch, each request's fields contiguous.  A request's future receives a
read-only mapping whose arrays are views of that array, made on access.

Each instance is solved by one thread block on the kernel path its own size selects, so a
request's result does not depend on what it was batched with.
"""
from __future__ import annotations

import collections
import collections.abc
import concurrent.futures
import ctypes
import dataclasses
import itertools
import threading
import time

import numpy as np
import torch

from . import _lib
from .qp import QP_F32, QP_F64, QPError, _check, default_options, workspace_bytes

GRAD_KEYS = ("dQ", "dq", "dG", "dh", "dA", "db")
# Field rules of qp_host_pack / qp_host_unpack (QP_FIELD_* in the C header).
F_Q, F_Q1, F_G, F_H, F_A, F_B = range(6)
# inputs Q, q, G, h, A, b and dℓ/dz; results z, λ, ν and the six gradients
FIELDS_IN = (F_Q, F_Q1, F_G, F_H, F_A, F_B, F_Q1)
FIELDS_OUT = (F_Q1, F_H, F_B, F_Q, F_Q1, F_G, F_H, F_A, F_B)
OUT_NAMES = ("z", "lam", "nu") + GRAD_KEYS


class ServedResult(collections.abc.Mapping):
    """Results of one request: z, lam, nu, the six gradients (views of the batch's result
    array, made on access) and the forward status."""

    __slots__ = ("_buf", "_off", "_dims", "status")

    def __init__(self, buf, off, dims, status):
        self._buf, self._off, self._dims, self.status = buf, int(off), dims, int(status)

    def _shapes(self):
        n, p, m = self._dims
        return ((n,), (p,), (m,), (n, n), (n,), (p, n), (p,), (m, n), (m,))

    def __getitem__(self, key):
        if key == "status":
            return self.status
        o = self._off
        for name, shp in zip(OUT_NAMES, self._shapes()):
            size = int(np.prod(shp))
            if name == key:
                return self._buf[o:o + size].reshape(shp)
            o += size
        raise KeyError(key)

    def __iter__(self):
        return iter(OUT_NAMES + ("status",))

    def __len__(self):
        return len(OUT_NAMES) + 1


@dataclasses.dataclass
class Request:
    data: tuple                 # (Q, q, G, h, A, b) host arrays
    dl_dz: np.ndarray
    arrival: float              # time.perf_counter() of arrival
    future: concurrent.futures.Future
    nbytes: int = 0
    stage_bytes: int = 0        # host staging bytes in its batch (set by submit)
    ptrs: tuple = ()            # host addresses of the six inputs and dl_dz (set by submit)

    @property
    def dims(self):
        Q, _, G, _, A, _ = self.data
        return (Q.shape[0], G.shape[0], A.shape[0])


def stage_bytes(dims, dtype=torch.float32) -> int:
    """Host staging bytes one request takes in its batch's pinned buffers: the larger of its
    packed inputs (with ∂ℓ/∂z*) and its packed results, plus its descriptor."""
    n, p, m = dims
    esz = 4 if dtype == torch.float32 else 8
    r4 = lambda x: (x + 3) // 4 * 4  # noqa: E731
    data = r4(n * n) + r4(n) + r4(p * n) + r4(p) + r4(m * n) + r4(m)
    return esz * max(data + r4(n), data + r4(n) + r4(p) + r4(m)) + 128


def request_bytes(dims, dtype=torch.float32) -> int:
    """Device bytes one request holds while in flight: its workspace plus its packed
    inputs, outputs and gradients (offsets padded to 4 elements)."""
    n, p, m = dims
    esz = 4 if dtype == torch.float32 else 8
    r4 = lambda x: (x + 3) // 4 * 4  # noqa: E731
    data = r4(n * n) + r4(n) + r4(p * n) + r4(p) + r4(m * n) + r4(m)
    return workspace_bytes(dtype, 1, n, p, m) + esz * (2 * data + 2 * r4(n) + r4(p) + r4(m)) + 64


class Admission:
    """Admission policy (host logic only): FIFO, a batch takes requests while the HBM budget,
    the batch-size cap and the staging cap allow; a request larger than the whole budget is
    rejected.  The staging cap bounds a batch's host staging bytes (``stage_bytes`` of its
    requests) so that it fits the stream slots' preallocated pinned buffers; a batch always
    takes at least one request."""

    def __init__(self, budget_bytes: int, max_batch: int, max_stage_bytes: int | None = None):
        self.budget = int(budget_bytes)
        self.max_batch = int(max_batch)
        self.max_stage = None if max_stage_bytes is None else int(max_stage_bytes)
        self.reserved = 0

    def take(self, queue: collections.deque):
        """Pop the next batch from ``queue``; returns (batch, rejected)."""
        batch, rejected, total, staged = [], [], 0, 0
        while queue and len(batch) < self.max_batch:
            r = queue[0]
            if r.nbytes > self.budget:
                rejected.append(queue.popleft())
                continue
            if self.reserved + total + r.nbytes > self.budget:
                break
            sb = getattr(r, "stage_bytes", 0)
            if batch and self.max_stage is not None and staged + sb > self.max_stage:
                break
            total += r.nbytes
            staged += sb
            batch.append(queue.popleft())
        self.reserved += total
        return batch, rejected, total

    def release(self, nbytes: int):
        self.reserved -= int(nbytes)


_FIELDS_IN_C = (ctypes.c_int32 * 7)(*FIELDS_IN)
_FIELDS_OUT_C = (ctypes.c_int32 * 9)(*FIELDS_OUT)


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
    # Defaults: the configuration measured best on a Poisson stream of n log-uniform in
    # [16, 512] (16 stream slots, size classes split at n = 64, 160 and 320, batches of at
    # most 256 requests).
    def __init__(self, device="cuda:0", dtype=torch.float32, max_inflight=16, max_batch=256,
                 hbm_budget_bytes=8 << 30, options=None, staging_bytes=32 << 20,
                 copy_threads=None, size_classes=(64, 160, 320)):
        self.device = torch.device(device)
        self.dtype = dtype
        self.options = options if options is not None else default_options(dtype)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(max_inflight)]
        import os
        self.copy_threads = int(copy_threads or min(8, os.cpu_count() or 1))
        esz = 4 if dtype == torch.float32 else 8
        self.staging = [_Staging(dtype, staging_bytes // esz) for _ in range(max_inflight)]
        self.stage_peak = (0, 0, 0)   # largest batch staging any slot has needed (elements)
        self.host_s = {"launch": 0.0, "retire": 0.0}
        self.phase_s = collections.defaultdict(float)   # host time by phase of _launch
        self.free_streams = list(range(max_inflight))
        # batches are capped to the slots' preallocated staging (less room for the per-field
        # section alignment), so that no slot grows its pinned buffers during a launch
        self.admission = Admission(hbm_budget_bytes, max_batch,
                                   max(staging_bytes - (64 << 10), 1 << 20))
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
        req.stage_bytes = stage_bytes(req.dims, self.dtype)
        req.ptrs = tuple(x.__array_interface__["data"][0] for x in data + (req.dl_dz,))
        with self.cv:
            n = req.dims[0]
            self.queues[sum(n >= t for t in self.size_classes)].append(req)
            self.cv.notify()
        return fut

    def equalize_staging(self, timeout=10.0):
        """Grow every stream slot's pinned staging to the largest any slot has needed so far.
        Slots grow on demand, so after a warm-up only the slots that carried its batches are
        large; a slot that grows later does so inside a batch's launch (a pinned allocation
        of tens of MB on the scheduler thread).  Call when no request is pending; it waits
        (up to `timeout` seconds) for the batches still in flight to retire."""
        deadline = time.perf_counter() + timeout
        while True:
            with self.cv:
                if not self.inflight and not any(self.queues):
                    for stg in self.staging:
                        stg.reserve(*self.stage_peak)
                    return
            if time.perf_counter() > deadline:
                raise RuntimeError("equalize_staging: the server did not become idle")
            time.sleep(1e-3)

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
        lib = _lib.load()
        stream, stg = self.streams[sidx], self.staging[sidx]
        ph = self.phase_s
        B = len(reqs)
        code = QP_F32 if self.dtype == torch.float32 else QP_F64
        esz = 4 if self.dtype == torch.float32 else 8
        dims = np.array([r.dims for r in reqs], dtype=np.int32)
        desc = (_lib.QPInstanceDesc * B)()
        sizes = _lib.QPPackedSizes()
        _check(lib.qp_packed_plan_ex(ctypes.byref(self.options), code, B,
                                     dims.ctypes.data_as(ctypes.c_void_p), None, None, desc,
                                     ctypes.byref(sizes)))
        t1 = time.perf_counter()
        ph["plan"] += t1 - t0
        tin = [sizes.nQ, sizes.nq, sizes.nG, sizes.nh, sizes.nA, sizes.nb, sizes.nq]
        tout = [sizes.nq, sizes.nh, sizes.nb, sizes.nQ, sizes.nq, sizes.nG, sizes.nh, sizes.nA,
                sizes.nb]
        dbytes = B * ctypes.sizeof(_lib.QPInstanceDesc)
        isec, n_in = _sections(tin + [(dbytes + esz - 1) // esz])
        osec, n_out = _sections(tout)
        stg.reserve(n_in, n_out, B)
        self.stage_peak = (max(self.stage_peak[0], n_in), max(self.stage_peak[1], n_out),
                           max(self.stage_peak[2], B))
        # the descriptors travel in the same staging buffer, after the inputs
        ctypes.memmove(stg.inp.data_ptr() + isec[7] * esz, desc, dbytes)
        src = (ctypes.c_void_p * (7 * B))(*itertools.chain.from_iterable(r.ptrs for r in reqs))
        _check(lib.qp_host_pack(B, desc, esz, 7, _FIELDS_IN_C, (ctypes.c_int64 * 8)(*isec), src,
                                stg.inp.data_ptr(), self.copy_threads))
        t2 = time.perf_counter()
        ph["pack"] += t2 - t1
        with torch.cuda.stream(stream):
            dev_in = torch.empty(n_in, dtype=self.dtype, device=self.device)
            dev_in.copy_(stg.inp[:n_in], non_blocking=True)
            dev_out = torch.empty(n_out, dtype=self.dtype, device=self.device)
            # status [B] and iters [B] (int32), then resid [B, 4] (FP64) 16-byte aligned
            small = torch.empty(4 * ((3 * B + 3) // 4) + 8 * B, dtype=torch.int32,
                                device=self.device)
            ws = torch.empty(max(int(sizes.ws_bytes), 256), dtype=torch.uint8, device=self.device)
            pi, po = dev_in.data_ptr(), dev_out.data_ptr()
            a = [ctypes.c_void_p(pi + isec[k] * esz) if tin[k] else None for k in range(7)]
            o = [ctypes.c_void_p(po + osec[k] * esz) if tout[k] else None for k in range(9)]
            dsc = ctypes.c_void_p(pi + isec[7] * esz)
            st_p = small.data_ptr()
            status = ctypes.c_void_p(st_p)
            iters = ctypes.c_void_p(st_p + 4 * B)
            resid = ctypes.c_void_p(st_p + 4 * 4 * ((3 * B + 3) // 4))   # 16-byte aligned
            sh = ctypes.c_void_p(stream.cuda_stream)
            _check(lib.qp_forward_packed(ctypes.byref(self.options), code, B, dsc,
                                         ctypes.byref(sizes), a[0], a[1], a[2], a[3], a[4], a[5],
                                         o[0], o[1], o[2], status, iters, resid,
                                         ctypes.c_void_p(ws.data_ptr()), ws.numel(), sh))
            _check(lib.qp_backward_packed(ctypes.byref(self.options), code, B, dsc,
                                          ctypes.byref(sizes), a[0], a[2], a[4],
                                          ctypes.c_void_p(ws.data_ptr()), ws.numel(), a[6],
                                          o[3], o[4], o[5], o[6], o[7], o[8], None, sh))
            stg.out[:n_out].copy_(dev_out, non_blocking=True)
            stg.status[:B].copy_(small[:B], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        t3 = time.perf_counter()
        ph["device"] += t3 - t2
        self.host_s["launch"] += t3 - t0
        return {"reqs": reqs, "desc": desc, "osec": osec, "n_out": n_out, "event": ev,
                "stream": sidx, "keep": (dev_in, dev_out, small, ws)}

    def _retire(self, item):
        t0 = time.perf_counter()
        lib = _lib.load()
        reqs, osec = item["reqs"], item["osec"]
        B = len(reqs)
        stg = self.staging[item["stream"]]
        esz = stg.out.element_size()
        hout = np.empty(item["n_out"], dtype=stg.out.numpy().dtype)
        off = np.empty(B + 1, dtype=np.int64)
        _check(lib.qp_host_unpack(B, item["desc"], esz, 9, _FIELDS_OUT_C,
                                  (ctypes.c_int64 * 9)(*osec), ctypes.c_void_p(stg.out.data_ptr()),
                                  hout.ctypes.data_as(ctypes.c_void_p),
                                  off.ctypes.data_as(ctypes.c_void_p), self.copy_threads))
        status = stg.status[:B].numpy().copy()
        self.free_streams.append(item["stream"])   # the staging buffers are free again
        now = time.perf_counter()
        for i, r in enumerate(reqs):
            self.latencies.append(now - r.arrival)
            r.future.set_result(ServedResult(hout, off[i], r.dims, status[i]))
        self.completed += B
        self.admission.release(sum(r.nbytes for r in reqs))
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
