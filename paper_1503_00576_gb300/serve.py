"""Serving triangle counts: a request loop with continuous batching.

Requests (one graph each) arrive at any time.  A loop thread owns a few
persistent batch engines (tc_engine_*, each a CUDA-graph replay of the whole
pipeline on its own stream) and, whenever an engine is free, admits the
waiting requests that fit its capacity -- pairs, vertices, graphs: the HBM
it reserved at start-up -- as one batch, in arrival order.  Requests that
arrive while batches are on the GPU join the next free engine, so work from
different batches overlaps on the device.  Every request gets exactly the
count of its graph alone: a batch is counted as the disjoint union of its
graphs.

Admission control:
* a request whose graph needs more than an engine's capacity is refused
  (its future raises TCError with TC_ERR_OVERFLOW);
* ids are checked on the device, per graph: a request with an id out of
  range fails alone (TC_ERR_ID_RANGE) and the rest of its batch is exact;
* graphs registered with `register` stay on the device; their total size is
  bounded by the resident-store budget (refusals raise TC_ERR_OOM).

Latency is measured per request from `submit` to the moment its result is
set; `stats()` reports p50/p99 next to throughput.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import threading
import time

import numpy as np

from . import (TC_COUNT_ERROR, TC_ERR_ID_RANGE, TC_ERR_OOM, TC_ERR_OVERFLOW, Engine, TCError,
               _torch)
from .batching import Capacity


class _Req:
    __slots__ = ("src", "dst", "n", "pairs", "on_host", "future", "t_submit", "t_done")

    def __init__(self, src, dst, n, pairs, on_host, t_submit):
        self.src, self.dst, self.n, self.pairs, self.on_host = src, dst, n, pairs, on_host
        self.future = cf.Future()
        self.t_submit = t_submit
        self.t_done = None


class Server:
    """Continuous-batching triangle-count server on one GPU."""

    def __init__(self, cap: Capacity = Capacity(pairs=1 << 26, vertices=1 << 23, graphs=1024),
                 engines: int = 2, tuning=None, store_bytes: int = 8 << 30, device=None):
        torch = _torch()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self.cap = cap
        with torch.cuda.device(self.device):
            self.engines = [Engine(cap.pairs, cap.vertices, cap.graphs, tuning=tuning)
                            for _ in range(max(1, engines))]
        self.store_bytes = store_bytes
        self._resident = {}
        self._resident_bytes = 0
        self._next_handle = 1
        self._queue = collections.deque()
        self._cv = threading.Condition()
        self._stop = False
        self._done = []  # finished requests (for stats)
        self._outstanding = 0  # admitted, result not yet set
        self._t0 = None
        self._batches = 0
        self._thread = threading.Thread(target=self._loop, name="tc-serve", daemon=True)
        self._thread.start()

    # ------------------------------------------------------------ requests
    def _admit(self, req: _Req) -> cf.Future:
        if req.pairs > self.cap.pairs or req.n > self.cap.vertices:
            req.future.set_exception(TCError(TC_ERR_OVERFLOW, "graph of %d pairs and %d vertices "
                                             "exceeds an engine (%d, %d)" % (
                                                 req.pairs, req.n, self.cap.pairs,
                                                 self.cap.vertices)))
            return req.future
        with self._cv:
            if self._t0 is None:
                self._t0 = req.t_submit
            self._outstanding += 1
            self._queue.append(req)
            self._cv.notify()
        return req.future

    def submit(self, src, dst, n: int) -> cf.Future:
        """Count the triangles of the graph (src[i], dst[i]) on ids [0, n).

        src/dst: host int32 arrays (numpy, or CPU tensors; page-locked
        tensors are used in place, anything else is copied to page-locked
        memory so that the engine's host-to-device copy runs asynchronously).
        Returns a future of the count (int)."""
        t_submit = time.perf_counter()
        torch = _torch()
        if isinstance(src, torch.Tensor):
            if src.is_cuda or dst.is_cuda:
                raise TypeError("submit takes host arrays; use register for device graphs")
            if src.dtype != torch.int32 or dst.dtype != torch.int32:
                raise TypeError("edge arrays must be int32")
            ts, td = src.contiguous(), dst.contiguous()
            s, d = ts.numpy(), td.numpy()
        else:
            s = np.ascontiguousarray(src, np.int32)
            d = np.ascontiguousarray(dst, np.int32)
            ts = td = None
        if s.shape != d.shape or s.ndim != 1:
            raise ValueError("src and dst must be 1-D and of equal length")
        if n < 0:
            raise ValueError("n < 0")
        # ids are checked on the device, per graph of the batch
        if ts is None or not ts.is_pinned():
            ts = torch.from_numpy(s).pin_memory()
            td = torch.from_numpy(d).pin_memory()
        elif not td.is_pinned():
            td = td.pin_memory()
        return self._admit(_Req(ts, td, int(n), len(s), True, t_submit))

    def register(self, src, dst, n: int) -> int:
        """Keep a graph on the device; returns a handle for submit_resident."""
        torch = _torch()
        s = np.ascontiguousarray(src, np.int32)
        d = np.ascontiguousarray(dst, np.int32)
        if len(s) and (min(s.min(), d.min()) < 0 or max(s.max(), d.max()) >= n):
            raise TCError(TC_ERR_ID_RANGE, "a vertex id is outside [0, %d)" % n)
        need = 8 * len(s)
        with self._cv:
            if self._resident_bytes + need > self.store_bytes:
                raise TCError(TC_ERR_OOM, "resident store full (%d of %d bytes)" % (
                    self._resident_bytes, self.store_bytes))
            self._resident_bytes += need
            h = self._next_handle
            self._next_handle += 1
        with torch.cuda.device(self.device):
            ds = torch.from_numpy(s).to(self.device)
            dd = torch.from_numpy(d).to(self.device)
            # engines run on their own non-blocking streams: the copy must be done
            torch.cuda.current_stream(self.device).synchronize()
            self._resident[h] = (ds, dd, int(n), need)
        return h

    def unregister(self, handle: int) -> None:
        s, d, n, need = self._resident.pop(handle)
        with self._cv:
            self._resident_bytes -= need

    def submit_resident(self, handle: int) -> cf.Future:
        t_submit = time.perf_counter()
        s, d, n, _ = self._resident[handle]
        return self._admit(_Req(s, d, n, s.numel(), False, t_submit))

    # ------------------------------------------------------------ loop
    def _take_batch(self):
        """Longest prefix of same-kind waiting requests that fits an engine."""
        batch, pairs, verts = [], 0, 0
        kind = self._queue[0].on_host
        while self._queue and len(batch) < self.cap.graphs:
            r = self._queue[0]
            if r.on_host != kind or pairs + r.pairs > self.cap.pairs or \
                    verts + r.n > self.cap.vertices:
                break
            batch.append(self._queue.popleft())
            pairs += r.pairs
            verts += r.n
        return batch, kind

    def _finish(self, reqs, totals=None, exc=None):
        now = time.perf_counter()
        for i, r in enumerate(reqs):
            r.t_done = now
            if exc is not None:
                r.future.set_exception(exc)
            elif int(totals[i]) == TC_COUNT_ERROR:
                r.future.set_exception(TCError(TC_ERR_ID_RANGE, "a vertex id is outside "
                                               "[0, %d)" % r.n))
            else:
                r.future.set_result(int(totals[i]))
            r.src = r.dst = None
        with self._cv:
            self._done.extend(reqs)
            self._outstanding -= len(reqs)
            self._cv.notify_all()

    def _loop(self):
        torch = _torch()
        torch.cuda.set_device(self.device)
        busy = {}
        while True:
            for i, reqs in list(busy.items()):
                eng = self.engines[i]
                if eng.poll():
                    try:
                        self._finish(reqs, eng.wait())
                    except TCError as e:
                        if getattr(e, "totals", None) is not None:
                            self._finish(reqs, e.totals)  # only some graphs failed
                        else:
                            self._finish(reqs, exc=e)
                    del busy[i]
            with self._cv:
                for i, eng in enumerate(self.engines):
                    if i in busy or not self._queue:
                        continue
                    batch, on_host = self._take_batch()
                    try:
                        eng.submit_parts([(r.src, r.dst, r.n) for r in batch], on_host)
                        busy[i] = batch
                        self._batches += 1
                    except TCError as e:
                        self._cv.release()
                        try:
                            self._finish(batch, exc=e)
                        finally:
                            self._cv.acquire()
                if self._stop and not busy and not self._queue:
                    return
                if not busy and not self._queue:
                    self._cv.wait(timeout=0.05)
                    continue
            if busy:
                time.sleep(5e-5)

    # ------------------------------------------------------------ control
    def drain(self, timeout: float = None) -> None:
        """Wait until every admitted request has its result."""
        with self._cv:
            if not self._cv.wait_for(lambda: self._outstanding == 0, timeout):
                raise TimeoutError("%d requests still pending" % self._outstanding)

    def close(self) -> None:
        with self._cv:
            self._stop = True
            self._cv.notify()
        self._thread.join()
        for e in self.engines:
            e.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def stats(self, reset: bool = False) -> dict:
        """p50/p99 latency (ms) and throughput of the requests finished so far."""
        with self._cv:
            done = list(self._done)
            t0 = self._t0
            batches = self._batches
            if reset:
                self._done, self._t0, self._batches = [], None, 0
        if not done:
            return {"requests": 0}
        lat = np.array([r.t_done - r.t_submit for r in done]) * 1e3
        span = max(r.t_done for r in done) - t0
        return {"requests": len(done), "batches": batches,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
                "graphs_per_s": len(done) / span if span > 0 else float("inf"),
                "span_s": span}


def poisson_stream(server: Server, graphs, rate: float, seed: int):
    """Submit graphs (list of (src, dst, n)) at seeded Poisson arrival times
    of the given rate (requests/s); returns the futures in order."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, len(graphs))
    t = time.perf_counter()
    futs = []
    for (s, d, n), gap in zip(graphs, gaps):
        t += gap
        while True:
            now = time.perf_counter()
            if now >= t:
                break
            time.sleep(min(t - now, 1e-3))
        futs.append(server.submit(s, d, n))
    return futs
