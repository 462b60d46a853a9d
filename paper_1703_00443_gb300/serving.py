"""Serving loop: continuous batching of forward+backward QP requests on one GPU.

Requests (Q, q, G, h, A, b, ∂ℓ/∂z*) of any sizes arrive at any time.  A scheduler thread
admits queued requests, oldest first, into a new packed batch whenever a stream slot is free
and the HBM budget covers the batch (workspace, packed inputs, outputs and gradients).  Each
admitted batch runs forward and backward (one persistent launch each, ``packed.PackedBatch``)
on its own CUDA stream, so a batch admitted while others are running overlaps with them on
the device; its iterates and factorisation stay in device memory between the two launches.
When a batch's completion event fires, its results are copied to the host, every request's
future is resolved with its own z*, λ*, ν* and gradients, and the batch's slot and budget are
released.  Latency is measured from each request's arrival to the resolution of its future.

Each instance is solved by one thread block on the kernel path its own size selects, so a
request's result does not depend on what it was batched with.
"""
from __future__ import annotations

import collections
import concurrent.futures
import dataclasses
import threading
import time

import numpy as np
import torch

from .packed import PackedBatch
from .qp import default_options, workspace_bytes

GRAD_KEYS = ("dQ", "dq", "dG", "dh", "dA", "db")


@dataclasses.dataclass
class Request:
    data: tuple                 # (Q, q, G, h, A, b) host arrays
    dl_dz: np.ndarray
    arrival: float              # time.perf_counter() of arrival
    future: concurrent.futures.Future
    nbytes: int = 0

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


class QPServer:
    def __init__(self, device="cuda:0", dtype=torch.float32, max_inflight=3, max_batch=1024,
                 hbm_budget_bytes=8 << 30, options=None):
        self.device = torch.device(device)
        self.dtype = dtype
        self.options = options if options is not None else default_options(dtype)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(max_inflight)]
        self.free_streams = list(range(max_inflight))
        self.admission = Admission(hbm_budget_bytes, max_batch)
        self.queue = collections.deque()
        self.cv = threading.Condition()
        self.inflight = []
        self.latencies = []
        self.batch_sizes = []
        self.completed = 0
        self._stop = False
        self._thread = threading.Thread(target=self._loop, daemon=True)
        self._thread.start()

    # ------------------------------------------------------------------ client side
    def submit(self, Q, q, G, h, A, b, dl_dz, arrival=None) -> concurrent.futures.Future:
        npdt = np.float32 if self.dtype == torch.float32 else np.float64
        data = tuple(np.ascontiguousarray(np.asarray(x), dtype=npdt) for x in (Q, q, G, h, A, b))
        fut = concurrent.futures.Future()
        req = Request(data, np.ascontiguousarray(np.asarray(dl_dz), dtype=npdt),
                      time.perf_counter() if arrival is None else arrival, fut)
        req.nbytes = request_bytes(req.dims, self.dtype)
        with self.cv:
            self.queue.append(req)
            self.cv.notify()
        return fut

    def close(self):
        with self.cv:
            self._stop = True
            self.cv.notify()
        self._thread.join()

    def stats(self):
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return {"completed": self.completed, "batches": len(self.batch_sizes),
                "mean_batch": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
                "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99))}

    # ------------------------------------------------------------------ scheduler
    def _launch(self, reqs, sidx):
        stream = self.streams[sidx]
        dims = [r.dims for r in reqs]
        with torch.cuda.stream(stream):
            pb = PackedBatch(dims, dtype=self.dtype, device=self.device, options=self.options)
            host = []
            for j, key in enumerate(pb.KEYS):
                buf = torch.zeros(max(pb.totals[key], 1), dtype=self.dtype).pin_memory()
                for o, l, r in zip(pb.offsets[key], pb.lengths[key], reqs):
                    if l:
                        buf[o:o + l] = torch.from_numpy(r.data[j].reshape(-1))
                host.append(buf)
            gbuf = torch.zeros(max(pb.totals["q"], 1), dtype=self.dtype).pin_memory()
            for o, l, r in zip(pb.offsets["q"], pb.lengths["q"], reqs):
                gbuf[o:o + l] = torch.from_numpy(r.dl_dz.reshape(-1))
            dev = [t.to(self.device, non_blocking=True) for t in host]
            g = gbuf.to(self.device, non_blocking=True)
            Q, q, G, h, A, b = dev
            out = pb.forward(Q, q, G, h, A, b)
            grads = pb.backward(Q, G, A, g)
            res = {"z": out.z.to("cpu", non_blocking=True), "lam": out.lam.to("cpu", non_blocking=True),
                   "nu": out.nu.to("cpu", non_blocking=True),
                   "status": out.status.to("cpu", non_blocking=True)}
            for k, t in zip(GRAD_KEYS, grads):
                res[k] = t.to("cpu", non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        return {"reqs": reqs, "pb": pb, "res": res, "event": ev, "stream": sidx,
                "keep": (host, gbuf, dev, g, out, grads)}

    def _retire(self, item):
        pb, res, reqs = item["pb"], item["res"], item["reqs"]
        now = time.perf_counter()
        views = {"z": pb.unpack(res["z"], "q"), "lam": pb.unpack(res["lam"], "h"),
                 "nu": pb.unpack(res["nu"], "b")}
        for k, key in zip(GRAD_KEYS, pb.KEYS):
            views[k] = pb.unpack(res[k], key)
        status = res["status"].numpy()
        for i, r in enumerate(reqs):
            out = {k: views[k][i].numpy().copy() for k in views}
            out["status"] = int(status[i])
            self.latencies.append(now - r.arrival)
            r.future.set_result(out)
        self.completed += len(reqs)
        self.admission.release(sum(r.nbytes for r in reqs))
        self.free_streams.append(item["stream"])

    def _loop(self):
        torch.cuda.set_device(self.device)
        while True:
            with self.cv:
                if self._stop and not self.queue and not self.inflight:
                    return
                if not self.queue and not self.inflight:
                    self.cv.wait(timeout=0.05)
            progressed = False
            # retire finished batches
            for item in list(self.inflight):
                if item["event"].query():
                    self.inflight.remove(item)
                    self._retire(item)
                    progressed = True
            # admit new batches while slots and budget allow
            while self.free_streams:
                with self.cv:
                    reqs, rejected, _ = self.admission.take(self.queue)
                for r in rejected:
                    r.future.set_exception(MemoryError(
                        f"request needs {r.nbytes} bytes, over the HBM budget {self.admission.budget}"))
                if not reqs:
                    break
                sidx = self.free_streams.pop(0)
                self.inflight.append(self._launch(reqs, sidx))
                self.batch_sizes.append(len(reqs))
                progressed = True
            if not progressed:
                time.sleep(5e-5)


def poisson_run(server: QPServer, pool, rate: float, count: int, seed: int = 0):
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
            if target - now > 2e-4:
                time.sleep(target - now - 1e-4)
        data, g = pool[k % len(pool)]
        futs.append(server.submit(*data, g, arrival=target))
    results = [f.result() for f in futs]
    return results, time.perf_counter() - t0
