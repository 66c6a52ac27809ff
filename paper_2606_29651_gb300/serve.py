"""Continuous-batching server for orbit-count requests.

Requests (one graph each, CSR in host memory) arrive at any time. Each of
`streams` worker threads owns a CUDA stream and its pinned staging buffers;
a free worker admits the waiting requests in arrival order while their
device footprint fits a memory budget, packs them into one
niorca_count_batch call on its stream, waits for it, and hands out the
counts. Graphs that arrive while the workers are busy join the next batch,
and one worker's packing and copying out overlap with the others' batches on
the GPU (no worker waits on another's host work). A request's latency runs
from submit() to the moment its counts are in host memory.

The counts of a graph do not depend on which other graphs share its batch
(the batched call counts the disjoint union, and no graphlet spans two
components), so every result is identical alone and in the mix. Each batch
reads the status word of its own stream. When a batch of several requests
reports a malformed graph, its requests are queued again, each to run alone,
so that only the malformed one fails.
"""
from __future__ import annotations

import collections
import os
import threading
import time
from concurrent.futures import Future, ThreadPoolExecutor

import numpy as np
import torch

from . import _lib


class Request:
    __slots__ = ("rowptr", "colidx", "n", "m", "future", "t_submit", "t_done", "alone")

    def __init__(self, rowptr: np.ndarray, colidx: np.ndarray):
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        self.colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        self.n = len(self.rowptr) - 1
        self.m = len(self.colidx)
        self.future: Future = Future()
        self.t_submit = time.perf_counter()
        self.t_done = None
        self.alone = False   # run in a batch of its own (after its batch failed)


def footprint(num_graphs: int, total_n: int, total_m: int) -> int:
    """Device bytes one batch holds while in flight: CSR, offsets, output and
    the library's work memory."""
    io = 4 * (total_n + 1) + 4 * total_m + 16 * (num_graphs + 1) + 120 * total_n
    return io + _lib.batch_workspace_bytes(num_graphs, total_n, total_m)


class _Slot:
    """A stream and its pinned host staging buffers, kept from batch to batch
    (pinning memory is far slower than copying into it); a buffer grows by
    half again when a batch needs more."""

    def __init__(self, stream):
        self.stream = stream
        self._bufs = {}

    def host(self, name: str, numel: int, dtype) -> torch.Tensor:
        buf = self._bufs.get(name)
        if buf is None or buf.numel() < numel:
            size = max(numel, int(1.5 * buf.numel()) if buf is not None else numel, 1)
            buf = torch.empty(size, dtype=dtype).pin_memory()
            self._bufs[name] = buf
        return buf[:numel]


class _Batch:
    def __init__(self, reqs, slot, nbytes):
        self.reqs = reqs
        self.slot = slot
        self.stream = slot.stream
        self.nbytes = nbytes
        self.event = torch.cuda.Event()
        self.host_out = None
        self.keep = None


class Server:
    """Continuous batching over `streams` CUDA streams within `mem_budget` bytes.

    Each stream has a worker thread; batches pack their CSR and copy out
    their counts on a small shared thread pool when large. A request's
    result is an int64 [n, 15] view of its batch's array.
    """

    PARALLEL_ENTRIES = 1 << 19   # CSR entries (or count words) from which a batch uses the pool

    def __init__(self, device: int | torch.device = 0, mem_budget: int = 8 << 30, streams: int = 3,
                 max_batch_graphs: int = 4096, max_batch_edges: int = 64 << 20):
        self.device = torch.device("cuda", device) if isinstance(device, int) else device
        self.mem_budget = int(mem_budget)
        self.max_batch_graphs = int(max_batch_graphs)
        self.max_batch_edges = int(max_batch_edges)
        with torch.cuda.device(self.device):
            self.streams = [torch.cuda.Stream(self.device) for _ in range(streams)]
        self._pending: collections.deque = collections.deque()
        self._in_use = 0
        self._cv = threading.Condition()
        self._stop = False
        self.completed = 0
        self.batches = 0
        self._pool = ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1)),
                                        thread_name_prefix="niorca-pack")
        self._workers = [threading.Thread(target=self._work, args=(_Slot(st),), name=f"niorca-stream{i}",
                                          daemon=True) for i, st in enumerate(self.streams)]
        for t in self._workers:
            t.start()

    # -------------------------------------------------------------- client
    def submit(self, rowptr: np.ndarray, colidx: np.ndarray) -> Future:
        """Queue one graph; the future resolves to its int64 [n, 15] counts."""
        r = Request(rowptr, colidx)
        r.future.request = r   # submit / completion times for latency statistics
        if footprint(1, max(r.n, 1), r.m) > self.mem_budget:
            r.future.set_exception(_lib.NiorcaError(_lib.Status.ENOMEM, "request larger than the memory budget"))
            return r.future
        with self._cv:
            if self._stop:
                raise RuntimeError("server is shut down")
            self._pending.append(r)
            self._cv.notify()
        return r.future

    def shutdown(self, wait: bool = True) -> None:
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        if wait:
            for t in self._workers:
                t.join()
            self._pool.shutdown(wait=True)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.shutdown()

    # ------------------------------------------------------------- workers
    def _admit(self):
        """Pop the longest prefix of the queue that fits the free memory
        (called with the lock held)."""
        take, n, m = [], 0, 0
        while self._pending and len(take) < self.max_batch_graphs:
            r = self._pending[0]
            if take and (r.alone or take[0].alone):
                break
            need = footprint(len(take) + 1, n + r.n, m + r.m)
            if take and (need > self.mem_budget - self._in_use or m + r.m > self.max_batch_edges):
                break
            if not take and need > self.mem_budget - self._in_use:
                break            # wait for memory to free up
            take.append(self._pending.popleft())
            n += r.n
            m += r.m
        return take, footprint(len(take), n, m) if take else 0

    def _work(self, slot):
        torch.cuda.set_device(self.device)
        while True:
            with self._cv:
                while True:
                    reqs, nbytes = self._admit() if self._pending else ([], 0)
                    if reqs:
                        self._in_use += nbytes
                        self.batches += 1
                        break
                    if self._stop and not self._pending:
                        return
                    self._cv.wait(timeout=0.05)
            try:
                b = self._launch(slot, reqs, nbytes)
                b.event.synchronize()
                self._retire(b, time.perf_counter())
            except Exception as e:   # the call itself failed (e.g. no device memory)
                for r in reqs:
                    if not r.future.done():
                        r.t_done = time.perf_counter()
                        r.future.set_exception(e)
            with self._cv:
                self._in_use -= nbytes
                self._cv.notify_all()   # memory is free again

    def _launch(self, slot, reqs, nbytes):
        stream = slot.stream
        b = _Batch(reqs, slot, nbytes)
        ns = np.array([r.n for r in reqs], dtype=np.int64)
        ms = np.array([r.m for r in reqs], dtype=np.int64)
        vo = np.zeros(len(reqs) + 1, dtype=np.int64)
        eo = np.zeros(len(reqs) + 1, dtype=np.int64)
        vo[1:] = np.cumsum(ns)
        eo[1:] = np.cumsum(ms)
        total_n, total_m = int(vo[-1]), int(eo[-1])
        rowptr = slot.host("rowptr", total_n + 1, torch.int32)
        colidx = slot.host("colidx", max(total_m, 1), torch.int32)
        offs = slot.host("offs", 2 * (len(reqs) + 1), torch.int64)
        host_out = slot.host("out", total_n * 15, torch.int64).view(total_n, 15)
        rp, ci = rowptr.numpy(), colidx.numpy()

        def pack(lo, hi):
            for g in range(lo, hi):
                r = reqs[g]
                np.add(r.rowptr[:-1], np.int32(eo[g]), out=rp[vo[g]:vo[g + 1]])
                ci[eo[g]:eo[g + 1]] = r.colidx

        self._runs(pack, eo)
        rp[-1] = total_m
        offs.numpy()[:] = np.concatenate([vo, eo])
        with torch.cuda.stream(stream):
            d_rp = rowptr.to(self.device, non_blocking=True)
            d_ci = colidx[:total_m].to(self.device, non_blocking=True)
            d_off = offs.to(self.device, non_blocking=True)
            out = torch.empty((total_n, 15), dtype=torch.int64, device=self.device)
            _lib.count_batch(d_rp, d_ci, d_off[:len(reqs) + 1], d_off[len(reqs) + 1:], out, stream=stream)
            host_out.copy_(out, non_blocking=True)
            b.event.record(stream)
        b.host_out = host_out
        b.keep = (d_rp, d_ci, d_off, out, vo)
        return b

    def _runs(self, fn, offsets):
        """fn(lo, hi) over the requests of a batch; a batch with many entries
        (offsets: their prefix sums) is cut into runs of about equal size
        that run on the thread pool (numpy copies release the interpreter
        lock)."""
        count, total = len(offsets) - 1, int(offsets[-1])
        if total < self.PARALLEL_ENTRIES or count < 2:
            fn(0, count)
            return
        parts = self._pool._max_workers
        cuts = np.searchsorted(offsets, np.linspace(0, total, parts + 1)[1:-1])
        bounds = [0, *sorted(set(int(c) for c in cuts) - {0, count}), count]
        list(self._pool.map(lambda ab: fn(*ab), zip(bounds[:-1], bounds[1:])))

    def _ranges(self, fn, count, words):
        """fn(lo, hi) over [0, count) in equal ranges on the thread pool when
        the batch moves many words."""
        if words < self.PARALLEL_ENTRIES or count < 2:
            fn(0, count)
            return
        parts = self._pool._max_workers
        bounds = [count * k // parts for k in range(parts + 1)]
        list(self._pool.map(lambda k: fn(bounds[k], bounds[k + 1]), range(parts)))

    def _retire(self, b: _Batch, now: float):
        vo = b.keep[-1]
        err = None
        try:
            _lib.check(b.stream)
        except _lib.NiorcaError as e:
            err = e
        if err is None:
            # one array per batch, filled from the staging buffer by a copy
            # split into equal row ranges; every request gets a view of it
            res = b.host_out.numpy()
            total_n = int(vo[-1])
            out = np.empty((total_n, 15), dtype=np.int64)

            def unpack(lo, hi):
                out[lo:hi] = res[lo:hi]

            self._ranges(unpack, total_n, 15 * total_n)
        b.keep = None
        if err is not None and len(b.reqs) > 1 and err.status != _lib.Status.ECUDA:
            # a malformed graph fails the whole batch: run each request alone
            with self._cv:
                for r in reversed(b.reqs):
                    r.alone = True
                    self._pending.appendleft(r)
                self._cv.notify_all()
            return
        for g, r in enumerate(b.reqs):
            r.t_done = now
            if err is not None:
                r.future.set_exception(err)
            else:
                r.future.set_result(out[vo[g]:vo[g + 1]])
        with self._cv:
            self.completed += len(b.reqs)


def latency_stats(requests_latency_s) -> dict:
    a = np.sort(np.asarray(requests_latency_s, dtype=np.float64))
    if len(a) == 0:
        return {"p50_ms": None, "p99_ms": None}
    return {"p50_ms": float(np.percentile(a, 50) * 1e3), "p99_ms": float(np.percentile(a, 99) * 1e3),
            "mean_ms": float(a.mean() * 1e3), "max_ms": float(a.max() * 1e3)}
