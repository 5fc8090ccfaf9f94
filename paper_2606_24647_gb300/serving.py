"""Serving loop: continuous batching of fragment queries over resident dimension
tables, under a device-memory admission budget.

The paper's worker keeps data on the GPU across operators and throttles what is
in flight with flow control on the exchange (Sec. 3.3.2), and drives its
communication from one host thread (Sec. 3.3.3). This module is the single-GPU
counterpart for many concurrent queries: one host thread admits arriving
fragment queries in FIFO order while their working memory fits the budget,
launches everything admitted as ONE fused batch (px_fragments_run) whenever the
GPU is free, and completes a batch's queries when its CUDA event fires. The
dimension tables stay resident; each query names one and brings its probe batch.

A query's result is the same whether it runs alone or in any mix: fragments of
a batch share no state (each has its own accumulators and outputs).
"""
from __future__ import annotations

import collections
import math
import time

import numpy as np
import torch

from . import PX_COUNT, PX_SUM, PX_SUM_MUL, FragmentBatch, Workspace, load


def poisson_arrivals(rate_qps: float, n: int, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of n queries of a Poisson process."""
    g = np.random.Generator(np.random.PCG64(seed))
    if rate_qps == math.inf:
        return np.zeros(n)
    return np.cumsum(g.exponential(1.0 / rate_qps, size=n))


def percentiles(lat_s) -> dict:
    a = np.asarray(lat_s, dtype=np.float64)
    if a.size == 0:
        return {"p50_ms": None, "p99_ms": None, "mean_ms": None}
    return {"p50_ms": float(np.percentile(a, 50) * 1e3), "p99_ms": float(np.percentile(a, 99) * 1e3),
            "mean_ms": float(a.mean() * 1e3)}


class Admission:
    """FIFO admission under a byte budget: a query is admitted only when its bytes
    fit next to everything in flight, and never ahead of an earlier waiting query."""

    def __init__(self, budget: int):
        self.budget = int(budget)
        self.used = 0
        self.peak = 0

    def fits(self, nbytes: int) -> bool:
        return self.used + nbytes <= self.budget

    def admit(self, nbytes: int) -> None:
        if nbytes > self.budget:
            raise ValueError(f"query of {nbytes} bytes can never fit the {self.budget}-byte budget")
        if not self.fits(nbytes):
            raise RuntimeError("admission over budget")
        self.used += nbytes
        self.peak = max(self.peak, self.used)

    def release(self, nbytes: int) -> None:
        self.used -= nbytes
        if self.used < 0:
            raise RuntimeError("released more than admitted")


class ResidentDim:
    """A resident dimension table: pk (int64), the group attribute (int32, values
    0..ngroups-1) and its unique join table, built once."""

    def __init__(self, pk: torch.Tensor, attr: torch.Tensor, ngroups: int, ws: Workspace | None = None):
        from . import px_join_build
        L = load()
        self.pk, self.attr, self.ngroups = pk, attr, int(ngroups)
        self.table = torch.empty(L.px_join_table_bytes(max(1, pk.numel()), 0), dtype=torch.uint8, device=pk.device)
        px_join_build([pk, attr], 0, unique=True, pay_col=1, table=self.table, ws=ws)


class Query:
    """One fragment query: filter date in [lo, hi) on its probe batch, join key = the
    named dimension's pk, group by dimension attr: SUM(price), SUM(price*qty), COUNT."""

    __slots__ = ("qid", "dim", "cols", "lo", "hi", "arrival", "admitted", "done", "out", "nbytes", "prepared")

    def __init__(self, qid: int, dim: ResidentDim, cols: dict, lo: int, hi: int):
        self.qid, self.dim, self.cols, self.lo, self.hi = qid, dim, cols, lo, hi
        self.arrival = self.admitted = self.done = None
        self.out = None
        self.prepared = None
        n = int(cols["key"].numel())
        g = dim.ngroups
        # working memory charged while in flight: the probe batch, the dense
        # accumulators and flags, and the outputs
        self.nbytes = 28 * n + 25 * g + 28 * g

    def prepare(self) -> None:
        """Result buffers and the fused-batch descriptor, built once when the query
        is created (as a request carries its result buffer), so that forming a batch
        only copies descriptors."""
        from . import fragment_descriptor
        dev = self.cols["key"].device
        g = self.dim.ngroups
        self.out = (torch.empty(g, dtype=self.dim.attr.dtype, device=dev),
                    [torch.empty(g, dtype=torch.int64, device=dev) for _ in range(3)],
                    torch.zeros(1, dtype=torch.int64, device=dev))
        self.prepared = fragment_descriptor(self.fragment())

    def fragment(self) -> dict:
        c, d = self.cols, self.dim
        return {"key": c["key"], "filter": c["date"], "lo": self.lo, "hi": self.hi, "cols": [c["price"], c["qty"]],
                "aggs": [(PX_SUM, 0, None), (PX_SUM_MUL, 0, 1), (PX_COUNT, None, None)], "table": d.table,
                "group": d.attr, "group_lo": 0, "group_hi": d.ngroups - 1, "max_groups": d.ngroups,
                "out": self.out}


class Server:
    """Continuous-batching server on one GPU stream (see the module docstring).
    Up to two batches are in flight: the host forms and launches the next batch
    while the previous one runs, so the GPU does not wait for the host."""

    def __init__(self, budget_bytes: int, max_batch: int = 512, config: tuple | None = None, stream=None,
                 inflight: int = 2):
        self.adm = Admission(budget_bytes)
        self.max_batch = max_batch
        self.config = config
        self.stream = stream or torch.cuda.current_stream()
        self.depth = inflight
        L = load()
        self.plans = [torch.empty(L.px_fragments_plan_bytes(max_batch), dtype=torch.uint8).pin_memory()
                      for _ in range(inflight)]
        self.wss = [Workspace(1 << 24) for _ in range(inflight)]
        self.batches = 0

    def serve(self, queries: list, arrivals, clock=time.perf_counter) -> dict:
        """Serve queries arriving at `arrivals` (seconds from the start, ascending).
        Returns stats; each query gets .out, .arrival, .done (host seconds)."""
        waiting = collections.deque()
        nxt = 0
        inflight = collections.deque()  # (event, queries, slot) in launch order
        free_slots = list(range(self.depth))
        done = 0
        t0 = clock()
        while done < len(queries):
            now = clock() - t0
            while nxt < len(queries) and arrivals[nxt] <= now:
                q = queries[nxt]
                q.arrival = float(arrivals[nxt])
                waiting.append(q)
                nxt += 1
            while inflight and inflight[0][0].query():
                ev, batch, slot = inflight.popleft()
                t_done = clock() - t0
                for q in batch:
                    q.done = t_done
                    self.adm.release(q.nbytes)
                done += len(batch)
                free_slots.append(slot)
            if free_slots and waiting:
                batch = []
                while waiting and len(batch) < self.max_batch and self.adm.fits(waiting[0].nbytes):
                    q = waiting.popleft()
                    self.adm.admit(q.nbytes)
                    q.admitted = clock() - t0
                    if q.prepared is None:
                        q.prepare()
                    batch.append(q)
                if batch:
                    slot = free_slots.pop()
                    fb = FragmentBatch(None, config=self.config, ws=self.wss[slot], plan=self.plans[slot],
                                       prepared=[q.prepared for q in batch])
                    self.wss[slot] = fb.ws
                    fb.run(self.stream)
                    ev = torch.cuda.Event()
                    ev.record(self.stream)
                    inflight.append((ev, batch, slot))
                    self.batches += 1
                elif not inflight:
                    raise RuntimeError("a waiting query exceeds the admission budget")
            if not inflight and not waiting and nxt < len(queries):
                wait = arrivals[nxt] - (clock() - t0)
                if wait > 2e-4:
                    time.sleep(wait - 1e-4)
        elapsed = max(q.done for q in queries) if queries else 0.0
        lat = [q.done - q.arrival for q in queries]
        return {"queries": len(queries), "batches": self.batches, "elapsed_s": elapsed,
                "qps": len(queries) / elapsed if elapsed > 0 else None, "peak_admitted_bytes": self.adm.peak,
                **percentiles(lat)}


class OneAtATimeServer:
    """The same queries served one at a time, FIFO, each through the unfused calls
    (px_filter -> px_join_probe -> px_groupby_agg) as soon as the previous query
    finished."""

    def __init__(self, stream=None):
        from . import px_filter, px_groupby_agg, px_join_probe  # noqa: F401
        self.stream = stream or torch.cuda.current_stream()
        self.ws = Workspace(1 << 24)
        self.bufs = None

    def _run(self, q: Query):
        from . import px_filter, px_groupby_agg, px_join_probe
        L = load()
        c, d = q.cols, q.dim
        n = max(1, int(c["key"].numel()))
        dev = c["key"].device
        if self.bufs is None or self.bufs[0].numel() < n:
            self.bufs = (torch.empty(n, dtype=torch.int32, device=dev), torch.empty(1, dtype=torch.int64, device=dev),
                         [torch.empty(n, dtype=torch.int64, device=dev), torch.empty(n, dtype=torch.int64, device=dev),
                          torch.empty(n, dtype=torch.int32, device=dev)])
        sel, nsel, jout = self.bufs
        self.ws.ensure(max(L.px_filter_ws_bytes(n), L.px_join_probe_ws_bytes(n), L.px_groupby_ws_bytes(n, d.ngroups)))
        px_filter(c["date"], q.lo, q.hi, sel=sel, nsel=nsel, ws=self.ws, stream=self.stream)
        j = px_join_probe(d.table, [c["key"], c["price"], c["qty"]], 0, sel=sel, nsel=nsel, carry=[1, 2],
                          payload=[d.attr], out=jout, out_cap=jout[0].numel(), ws=self.ws, stream=self.stream)
        g = px_groupby_agg(jout, [2], [(PX_SUM, 0, None), (PX_SUM_MUL, 0, 1), (PX_COUNT, None, None)],
                           max_groups=d.ngroups, d_nrows=j["nout"], key_range=[(0, d.ngroups - 1)], ws=self.ws,
                           stream=self.stream)
        q.out = (g["keys"][0], g["aggs"], g["ngroups"])

    def serve(self, queries: list, arrivals, clock=time.perf_counter) -> dict:
        t0 = clock()
        for q, a in zip(queries, arrivals):
            now = clock() - t0
            if a > now + 2e-4:
                time.sleep(a - now - 1e-4)
            q.arrival = float(a)
            self._run(q)
            self.stream.synchronize()
            q.done = clock() - t0
        elapsed = max(q.done for q in queries) if queries else 0.0
        lat = [q.done - q.arrival for q in queries]
        return {"queries": len(queries), "elapsed_s": elapsed, "qps": len(queries) / elapsed if elapsed > 0 else None,
                **percentiles(lat)}
