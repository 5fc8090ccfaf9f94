"""The three operator pipelines of the workloads, each a chain of px_* calls on one
stream with every buffer allocated once up front (so a step allocates nothing and
never synchronises with the host).

* PlainPipeline      - filter -> hash exchange -> group-by (a Q1-like scan-filter-
                       aggregate, Sec. 2.3), over one columnar batch.
* JoinPipeline       - filter -> join build -> join probe -> group-by (a Q5/Q9-like
                       filter-join-aggregate, Sec. 3.4).
* AtScalePipeline    - exchange of both join sides into P partitions -> per-partition
                       join build and probe -> Partial group-by per partition -> Final
                       merge (the exchange feeding the join and aggregation, Sec. 3.3
                       with the aggregation modes of Sec. 3.2).
* WideJoinPipeline   - a selective join over a wide fact, eager (exchange every needed
                       column) or late-materialized (exchange (key, row id), gather the
                       payload after the join; Sec. 2.3).
* StreamingAggregation - Partial aggregation over a stream of batches emitting its
                       groups into a Final aggregation past a size threshold (Sec. 3.2).
* FragmentSet        - many small filter -> join -> aggregate fragments over resident
                       dimension tables, run as one fused batch (px_fragments_run);
  OneAtATime         - the same fragments one at a time through the unfused calls.
"""
from __future__ import annotations

import torch

from . import (PX_AGG_ACCUMULATE, PX_AGG_STREAM, PX_COUNT, PX_SUM, PX_SUM_MUL, FragmentBatch, Workspace, load,
               px_filter, px_gather, px_groupby_agg, px_join_build, px_join_probe, px_join_probe_agg, px_partition)


def _empty_like_cols(cols, n=None):
    return [torch.empty(max(n if n is not None else c.numel(), 1), dtype=c.dtype, device=c.device) for c in cols]


class PlainPipeline:
    """date filter -> partition on key -> group by (flag, status): SUM(price),
    SUM(price*qty), SUM(qty), COUNT(*)."""

    NAMES = ["key", "price", "qty", "date", "flag", "status"]

    def __init__(self, d: dict, lo: int, hi: int, nparts: int = 8, seed: int = 0, max_groups: int = 256,
                 key_range=((0, 3), (0, 1))):
        L = load()
        self.d = d
        self.lo, self.hi, self.nparts, self.seed, self.max_groups = lo, hi, nparts, seed, max_groups
        self.key_range = key_range  # catalog statistic of (flag, status); speed only
        n = d["key"].numel()
        dev = d["key"].device
        self.cols = [d[k] for k in self.NAMES]
        self.sel = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        self.nsel = torch.empty(1, dtype=torch.int64, device=dev)
        self.parts = _empty_like_cols(self.cols)
        self.offsets = torch.empty(nparts + 1, dtype=torch.int64, device=dev)
        self.gout = [torch.empty(max_groups, dtype=torch.int8, device=dev) for _ in range(2)] + \
                    [torch.empty(max_groups, dtype=torch.int64, device=dev) for _ in range(4)]
        need = max(L.px_filter_ws_bytes(n), L.px_partition_ws_bytes(n, nparts), L.px_groupby_ws_bytes(n, max_groups))
        self.ws = Workspace(need)

    CALLS = ["px_filter", "px_partition", "px_groupby_agg"]

    def steps(self, stream=None) -> list:
        """The pipeline's calls in order, as (name, thunk) pairs; run() calls them all."""
        res = {}

        def groupby():
            res["groups"] = px_groupby_agg(
                self.parts, [4, 5], [(PX_SUM, 1, None), (PX_SUM_MUL, 1, 2), (PX_SUM, 2, None), (PX_COUNT, None, None)],
                max_groups=self.max_groups, d_nrows=self.nsel, key_range=self.key_range, out=self.gout, ws=self.ws,
                stream=stream)

        self._res = res
        return list(zip(self.CALLS, [
            lambda: px_filter(self.d["date"], self.lo, self.hi, sel=self.sel, nsel=self.nsel, ws=self.ws,
                              stream=stream),
            lambda: px_partition(self.cols, 0, self.nparts, self.seed, sel=self.sel, nsel=self.nsel, out=self.parts,
                                 offsets=self.offsets, ws=self.ws, stream=stream),
            groupby]))

    def run(self, stream=None) -> dict:
        for _, f in self.steps(stream):
            f()
        return {"sel": self.sel, "nsel": self.nsel, "parts": dict(zip(self.NAMES, self.parts)),
                "offsets": self.offsets, "groups": self._res["groups"]}


class JoinPipeline:
    """fact.date filter -> build on dim.pk -> probe fact.fk (carry amount, gather
    dim.attr) -> group by attr: SUM(amount), COUNT(*)."""

    def __init__(self, d: dict, lo: int, hi: int, max_groups: int = 64, attr_range=(0, 24)):
        L = load()
        self.d = d
        self.lo, self.hi, self.max_groups = lo, hi, max_groups
        self.attr_range = attr_range  # catalog statistic of dim.attr; speed only
        nf, nd = d["fk"].numel(), d["pk"].numel()
        dev = d["fk"].device
        self.fact = [d["fk"], d["amount"], d["date"]]
        self.dim = [d["pk"], d["attr"]]
        self.sel = torch.empty(max(nf, 1), dtype=torch.int32, device=dev)
        self.nsel = torch.empty(1, dtype=torch.int64, device=dev)
        self.table = torch.empty(L.px_join_table_bytes(nd, 0), dtype=torch.uint8, device=dev)
        self.jout = [torch.empty(max(nf, 1), dtype=torch.int64, device=dev),
                     torch.empty(max(nf, 1), dtype=torch.int32, device=dev)]
        self.gout = [torch.empty(max_groups, dtype=torch.int32, device=dev)] + \
                    [torch.empty(max_groups, dtype=torch.int64, device=dev) for _ in range(2)]
        need = max(L.px_filter_ws_bytes(nf), L.px_join_build_ws_bytes(nd), L.px_join_probe_ws_bytes(nf),
                   L.px_groupby_ws_bytes(nf, max_groups))
        self.ws = Workspace(need)

    CALLS = ["px_filter", "px_join_build", "px_join_probe", "px_groupby_agg"]

    def steps(self, stream=None) -> list:
        """The pipeline's calls in order, as (name, thunk) pairs; run() calls them all."""
        res = {}

        def probe():
            res["join"] = px_join_probe(self.table, self.fact, 0, sel=self.sel, nsel=self.nsel, carry=[1],
                                        payload=[self.d["attr"]], out=self.jout, out_cap=self.jout[0].numel(),
                                        ws=self.ws, stream=stream)

        def groupby():
            res["groups"] = px_groupby_agg(self.jout, [1], [(PX_SUM, 0, None), (PX_COUNT, None, None)],
                                           max_groups=self.max_groups, d_nrows=res["join"]["nout"],
                                           key_range=[self.attr_range] if self.attr_range else None, out=self.gout,
                                           ws=self.ws, stream=stream)

        self._res = res
        return list(zip(self.CALLS, [
            lambda: px_filter(self.d["date"], self.lo, self.hi, sel=self.sel, nsel=self.nsel, ws=self.ws,
                              stream=stream),
            lambda: px_join_build(self.dim, 0, unique=True, pay_col=1, table=self.table, ws=self.ws, stream=stream),
            probe, groupby]))

    def run(self, stream=None) -> dict:
        for _, f in self.steps(stream):
            f()
        return {"sel": self.sel, "nsel": self.nsel, "join": self._res["join"], "groups": self._res["groups"]}


class AtScalePipeline:
    """Exchange both sides on the join key into nparts partitions, join per partition,
    Partial group-by attr per partition (SUM(amount), COUNT(*)), Final merge by attr."""

    CALLS = ["px_partition(dim)", "px_partition(fact)", "px_join_build", "px_join_probe",
             "px_groupby_agg(partial)", "px_groupby_agg(final)"]
    CALLS_FUSED = ["px_partition(dim)", "px_partition(fact)", "px_join_build", "px_join_probe_agg(partial)",
                   "px_groupby_agg(final)"]

    def __init__(self, d: dict, nparts: int = 64, seed: int = 0, nattr_bound: int = 10_000, attr_range="auto",
                 fused: bool = False, fact_config=None, dim_config=None):
        L = load()
        self.d = d
        self.fused = fused  # probe + Partial group-by in one call (px_join_probe_agg)
        # launch shapes (items, blocks per SM) of the two exchanges, e.g. from
        # autotune.tune_partition; None = the library's defaults
        self.fact_config, self.dim_config = fact_config, dim_config
        self.nparts, self.seed = nparts, seed
        # catalog statistic of dim.attr (speed only); "auto": the attribute's domain [0, nattr_bound)
        self.attr_range = (0, nattr_bound - 1) if attr_range == "auto" else attr_range
        nf, nd = d["fk"].numel(), d["pk"].numel()
        dev = d["fk"].device
        self.fact = [d["fk"], d["amount"], d["date"]]
        self.dim = [d["pk"], d["attr"]]
        self.fparts = _empty_like_cols(self.fact)
        self.dparts = _empty_like_cols(self.dim)
        self.foff = torch.empty(nparts + 1, dtype=torch.int64, device=dev)
        self.doff = torch.empty(nparts + 1, dtype=torch.int64, device=dev)
        self.table = torch.empty(L.px_join_table_bytes(nd, nparts), dtype=torch.uint8, device=dev)
        self.jout = [torch.empty(max(nf, 1), dtype=torch.int64, device=dev),
                     torch.empty(max(nf, 1), dtype=torch.int32, device=dev)]
        self.max_partial = min(max(nf, 1), nparts * nattr_bound)
        self.max_final = min(max(nf, 1), nattr_bound)
        self.pout = [torch.empty(self.max_partial, dtype=torch.int32, device=dev)] + \
                    [torch.empty(self.max_partial, dtype=torch.int64, device=dev) for _ in range(2)]
        self.fout = [torch.empty(self.max_final, dtype=torch.int32, device=dev)] + \
                    [torch.empty(self.max_final, dtype=torch.int64, device=dev) for _ in range(2)]
        need = max(L.px_partition_ws_bytes(nf, nparts), L.px_partition_ws_bytes(nd, nparts),
                   L.px_join_build_ws_bytes(nd), L.px_join_probe_ws_bytes(nf),
                   L.px_groupby_ws_bytes(nf, self.max_partial), L.px_join_probe_agg_ws_bytes(nf, self.max_partial))
        self.ws = Workspace(need)

    def run(self, stream=None, mark=None) -> dict:
        if self.fused:
            return self._run_fused(stream, mark)
        """One pass of the pipeline. mark(i), if given, is called before call i and
        after the last one (i = 0..6), e.g. to record CUDA events between the calls."""
        P, ws = self.nparts, self.ws
        rng = [self.attr_range] if self.attr_range else None
        mark = mark or (lambda i: None)
        mark(0)
        px_partition(self.dim, 0, P, self.seed, out=self.dparts, offsets=self.doff, config=self.dim_config, ws=ws,
                     stream=stream)
        mark(1)
        px_partition(self.fact, 0, P, self.seed, out=self.fparts, offsets=self.foff, config=self.fact_config, ws=ws,
                     stream=stream)
        mark(2)
        px_join_build(self.dparts, 0, seg=self.doff, unique=True, pay_col=1, table=self.table, ws=ws,
                      stream=stream)
        mark(3)
        j = px_join_probe(self.table, self.fparts, 0, seg=self.foff, carry=[1], payload=[self.dparts[1]],
                          out=self.jout, out_cap=self.jout[0].numel(), out_seg=True, ws=ws, stream=stream)
        mark(4)
        part = px_groupby_agg(self.jout, [1], [(PX_SUM, 0, None), (PX_COUNT, None, None)],
                              max_groups=self.max_partial, seg=j["out_seg"], d_nrows=j["nout"], key_range=rng,
                              out=self.pout, ws=ws, stream=stream)
        mark(5)
        final = px_groupby_agg(self.pout, [0], [(PX_SUM, 1, None), (PX_SUM, 2, None)], max_groups=self.max_final,
                               d_nrows=part["ngroups"], key_range=rng, out=self.fout, ws=ws, stream=stream)
        mark(6)
        return {"dim_offsets": self.doff, "fact_offsets": self.foff, "join": j, "partial": part, "final": final}

    def _run_fused(self, stream=None, mark=None) -> dict:
        """The same pipeline with the probe and the Partial group-by fused
        (px_join_probe_agg): the joined rows are never written."""
        P, ws = self.nparts, self.ws
        lo, hi = self.attr_range
        mark = mark or (lambda i: None)
        mark(0)
        px_partition(self.dim, 0, P, self.seed, out=self.dparts, offsets=self.doff, config=self.dim_config, ws=ws,
                     stream=stream)
        mark(1)
        px_partition(self.fact, 0, P, self.seed, out=self.fparts, offsets=self.foff, config=self.fact_config, ws=ws,
                     stream=stream)
        mark(2)
        px_join_build(self.dparts, 0, seg=self.doff, unique=True, pay_col=1, table=self.table, ws=ws,
                      stream=stream)
        mark(3)
        part = px_join_probe_agg(self.table, self.fparts, 0, self.dparts[1], (lo, hi),
                                 [(PX_SUM, 1, None), (PX_COUNT, None, None)], max_groups=self.max_partial,
                                 seg=self.foff, out=self.pout, ws=ws, stream=stream)
        mark(4)
        rng = [self.attr_range]
        final = px_groupby_agg(self.pout, [0], [(PX_SUM, 1, None), (PX_SUM, 2, None)], max_groups=self.max_final,
                               d_nrows=part["ngroups"], key_range=rng, out=self.fout, ws=ws, stream=stream)
        mark(5)
        return {"dim_offsets": self.doff, "fact_offsets": self.foff, "partial": part, "final": final}


class FragmentSet:
    """Device-resident fragments of the batched workload: per fragment its fact
    columns, its dimension columns and its unique join table (built once, as a
    resident dimension table). Query of every fragment: keep date in [lo, hi),
    join key = pk, group by dim.attr (values 0..ngroups-1): SUM(price),
    SUM(price * qty), COUNT(*)."""

    def __init__(self, datas: list, ngroups: list, lo: int, hi: int, device=None, stream=None):
        L = load()
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.lo, self.hi = lo, hi
        self.ngroups = [int(g) for g in ngroups]
        self.cols, self.frags = [], []
        ws = Workspace(L.px_join_build_ws_bytes(1), device=dev)
        for d, ng in zip(datas, self.ngroups):
            c = {k: torch.from_numpy(d[k]).to(dev, non_blocking=True) for k in ("key", "price", "qty", "date", "pk", "attr")}
            c["table"] = torch.empty(L.px_join_table_bytes(max(1, d["pk"].size), 0), dtype=torch.uint8, device=dev)
            px_join_build([c["pk"], c["attr"]], 0, unique=True, pay_col=1, table=c["table"], ws=ws,
                          stream=stream)
            self.cols.append(c)
            self.frags.append({"key": c["key"], "filter": c["date"], "lo": lo, "hi": hi,
                               "cols": [c["price"], c["qty"]],
                               "aggs": [(PX_SUM, 0, None), (PX_SUM_MUL, 0, 1), (PX_COUNT, None, None)],
                               "table": c["table"], "group": c["attr"], "group_lo": 0, "group_hi": ng - 1,
                               "max_groups": ng})
        self.rows = sum(int(c["key"].numel()) for c in self.cols)

    def batch(self, idx=None, config=None, ws=None) -> FragmentBatch:
        frags = self.frags if idx is None else [self.frags[i] for i in idx]
        return FragmentBatch(frags, config=config, ws=ws)


class OneAtATime:
    """The same fragments run one at a time through the unfused calls
    (px_filter -> px_join_probe -> px_groupby_agg), every buffer allocated once
    and shared across fragments (they run in order on one stream)."""

    def __init__(self, fs: FragmentSet):
        L = load()
        self.fs = fs
        dev = fs.cols[0]["key"].device
        nmax = max(1, max(int(c["key"].numel()) for c in fs.cols))
        gmax = max(fs.ngroups)
        self.sel = torch.empty(nmax, dtype=torch.int32, device=dev)
        self.nsel = torch.empty(1, dtype=torch.int64, device=dev)
        self.jout = [torch.empty(nmax, dtype=torch.int64, device=dev), torch.empty(nmax, dtype=torch.int64, device=dev),
                     torch.empty(nmax, dtype=torch.int32, device=dev)]
        self.gout = [[torch.empty(g, dtype=torch.int32, device=dev)] +
                     [torch.empty(g, dtype=torch.int64, device=dev) for _ in range(3)] for g in fs.ngroups]
        need = max(L.px_filter_ws_bytes(nmax), L.px_join_probe_ws_bytes(nmax), L.px_groupby_ws_bytes(nmax, gmax))
        self.ws = Workspace(need, device=dev)
        self.results = [None] * len(fs.cols)

    def run(self, stream=None, idx=None):
        fs = self.fs
        for i in (range(len(fs.cols)) if idx is None else idx):
            c = fs.cols[i]
            px_filter(c["date"], fs.lo, fs.hi, sel=self.sel, nsel=self.nsel, ws=self.ws, stream=stream)
            j = px_join_probe(c["table"], [c["key"], c["price"], c["qty"]], 0, sel=self.sel, nsel=self.nsel,
                              carry=[1, 2], payload=[c["attr"]], out=self.jout, out_cap=self.jout[0].numel(),
                              ws=self.ws, stream=stream)
            ng = fs.ngroups[i]
            self.results[i] = px_groupby_agg(self.jout, [2], [(PX_SUM, 0, None), (PX_SUM_MUL, 0, 1),
                                                             (PX_COUNT, None, None)],
                                             max_groups=ng, d_nrows=j["nout"], key_range=[(0, ng - 1)],
                                             out=self.gout[i], ws=self.ws, stream=stream)
        return self.results


class WideJoinPipeline:
    """Selective join over a wide fact: exchange both sides into nparts partitions,
    join per partition, Partial group-by attr (SUM(amount), SUM(price*qty), COUNT)
    per partition, Final merge.

    late=False (eager): the fact exchange moves fk and every column the query needs
    after the join (amount, price, qty) and the probe carries them.
    late=True (late materialization, Sec. 2.3): the fact exchange moves only fk and a
    row id; the probe carries the row id, and px_gather fetches amount, price and
    qty for the rows that survived the join."""

    CALLS_EAGER = ["px_partition(dim)", "px_partition(fact)", "px_join_build", "px_join_probe",
                   "px_groupby_agg(partial)", "px_groupby_agg(final)"]
    CALLS_LATE = ["px_partition(dim)", "px_partition(fact)", "px_join_build", "px_join_probe", "px_gather",
                  "px_groupby_agg(partial)", "px_groupby_agg(final)"]

    def __init__(self, d: dict, late: bool, nparts: int = 64, seed: int = 0, nattr_bound: int = 1_000):
        L = load()
        self.d, self.late, self.nparts, self.seed = d, late, nparts, seed
        self.attr_range = (0, nattr_bound - 1)
        nf, nd = d["fk"].numel(), d["pk_b"].numel()
        dev = d["fk"].device
        self.rowid = torch.arange(nf, dtype=torch.int32, device=dev) if late else None
        self.fact = [d["fk"], self.rowid] if late else [d["fk"], d["amount"], d["price"], d["qty"]]
        self.dim = [d["pk_b"], d["attr_b"]]
        self.fparts = _empty_like_cols(self.fact)
        self.dparts = _empty_like_cols(self.dim)
        self.foff = torch.empty(nparts + 1, dtype=torch.int64, device=dev)
        self.doff = torch.empty(nparts + 1, dtype=torch.int64, device=dev)
        self.table = torch.empty(L.px_join_table_bytes(max(nd, 1), nparts), dtype=torch.uint8, device=dev)
        cap = max(nf, 1)
        if late:  # probe output: row id, attr; then the gathered payload
            self.jout = [torch.empty(cap, dtype=torch.int32, device=dev), torch.empty(cap, dtype=torch.int32, device=dev)]
            self.gout = [torch.empty(cap, dtype=torch.int64, device=dev) for _ in range(3)]
        else:     # probe output: amount, price, qty, attr
            self.jout = [torch.empty(cap, dtype=torch.int64, device=dev) for _ in range(3)] + \
                        [torch.empty(cap, dtype=torch.int32, device=dev)]
        self.max_partial = min(cap, nparts * nattr_bound)
        self.max_final = min(cap, nattr_bound)
        self.pout = [torch.empty(self.max_partial, dtype=torch.int32, device=dev)] + \
                    [torch.empty(self.max_partial, dtype=torch.int64, device=dev) for _ in range(3)]
        self.fout = [torch.empty(self.max_final, dtype=torch.int32, device=dev)] + \
                    [torch.empty(self.max_final, dtype=torch.int64, device=dev) for _ in range(3)]
        need = max(L.px_partition_ws_bytes(nf, nparts), L.px_partition_ws_bytes(nd, nparts),
                   L.px_join_build_ws_bytes(nd), L.px_join_probe_ws_bytes(nf),
                   L.px_groupby_ws_bytes(nf, self.max_partial))
        self.ws = Workspace(need)

    def run(self, stream=None, mark=None) -> dict:
        P, ws = self.nparts, self.ws
        rng = [self.attr_range]
        mark = mark or (lambda i: None)
        k = 0
        mark(k)
        px_partition(self.dim, 0, P, self.seed, out=self.dparts, offsets=self.doff, ws=ws, stream=stream)
        k += 1
        mark(k)
        px_partition(self.fact, 0, P, self.seed, out=self.fparts, offsets=self.foff, ws=ws, stream=stream)
        k += 1
        mark(k)
        px_join_build(self.dparts, 0, seg=self.doff, unique=True, pay_col=1, table=self.table, ws=ws,
                      stream=stream)
        k += 1
        mark(k)
        carry = [1] if self.late else [1, 2, 3]
        j = px_join_probe(self.table, self.fparts, 0, seg=self.foff, carry=carry, payload=[self.dparts[1]],
                          out=self.jout, out_cap=self.jout[0].numel(), out_seg=True, ws=ws, stream=stream)
        k += 1
        mark(k)
        if self.late:
            px_gather([self.d["amount"], self.d["price"], self.d["qty"]], self.jout[0], d_n=j["nout"],
                      out=self.gout, ws=ws, stream=stream)
            k += 1
            mark(k)
            cols = self.gout + [self.jout[1]]
        else:
            cols = self.jout
        part = px_groupby_agg(cols, [3], [(PX_SUM, 0, None), (PX_SUM_MUL, 1, 2), (PX_COUNT, None, None)],
                              max_groups=self.max_partial, seg=j["out_seg"], d_nrows=j["nout"], key_range=rng,
                              out=self.pout, ws=ws, stream=stream)
        k += 1
        mark(k)
        final = px_groupby_agg(self.pout, [0], [(PX_SUM, 1, None), (PX_SUM, 2, None), (PX_SUM, 3, None)],
                               max_groups=self.max_final, d_nrows=part["ngroups"], key_range=rng, out=self.fout,
                               ws=ws, stream=stream)
        k += 1
        mark(k)
        return {"join": j, "partial": part, "final": final}


class StreamingAggregation:
    """Partial aggregation over a stream of batches that emits its groups into a
    Final aggregation whenever they reach `threshold` (HashAggregation's Partial and
    Final modes, Sec. 3.2), all on one stream; the final result equals one Single
    aggregation over every batch fed. The size check is asynchronous: the group
    count of feed k is read (from pinned host memory) before feed k + 2, so the
    Partial table holds at most threshold + two batches' new groups
    (max_partial must allow that)."""

    def __init__(self, key_dtype, aggs: list, *, threshold: int, max_partial: int, max_final: int,
                 key_range=None, device=None):
        L = load()
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.aggs, self.threshold = aggs, int(threshold)
        self.max_partial, self.max_final, self.key_range = int(max_partial), int(max_final), key_range
        na = len(aggs)
        self.pout = [torch.empty(self.max_partial, dtype=key_dtype, device=dev)] + \
                    [torch.empty(self.max_partial, dtype=torch.int64, device=dev) for _ in range(na)]
        self.fout = [torch.empty(self.max_final, dtype=key_dtype, device=dev)] + \
                    [torch.empty(self.max_final, dtype=torch.int64, device=dev) for _ in range(na)]
        self.p_ng = torch.zeros(1, dtype=torch.int64, device=dev)
        self.f_ng = torch.zeros(1, dtype=torch.int64, device=dev)
        self.ws_p = Workspace(L.px_groupby_ws_bytes(1, self.max_partial), device=dev)
        self.ws_f = Workspace(L.px_groupby_ws_bytes(1, self.max_final), device=dev)
        self.host_counts = [torch.zeros(1, dtype=torch.int64).pin_memory() for _ in range(2)]
        self.events = [None, None]
        self.partial_fresh = True
        self.final_fresh = True
        self.feeds = 0
        self.emissions = 0

    def feed(self, cols: list, key_col: int, d_nrows=None, stream=None):
        """Aggregate one batch (cols[key_col] the key) into the Partial stream."""
        k = self.feeds % 2
        ev = self.events[k]  # the count copied two feeds ago
        if ev is not None:
            ev.synchronize()
            self.events[k] = None
            if not self.partial_fresh and int(self.host_counts[k].item()) >= self.threshold:
                self.emit(stream)
        px_groupby_agg(cols, [key_col], self.aggs, max_groups=self.max_partial, d_nrows=d_nrows,
                       key_range=self.key_range, out=self.pout, ws=self.ws_p, stream=stream, ngroups=self.p_ng,
                       flags=PX_AGG_STREAM if self.partial_fresh else PX_AGG_ACCUMULATE)
        self.partial_fresh = False
        s = stream or torch.cuda.current_stream()
        self.host_counts[k].copy_(self.p_ng, non_blocking=True)
        e = torch.cuda.Event()
        e.record(s)
        self.events[k] = e
        self.feeds += 1

    def emit(self, stream=None):
        """Merge the Partial groups into the Final stream and restart the Partial."""
        if self.partial_fresh:
            return
        rng = [self.key_range[0]] if self.key_range else None
        px_groupby_agg(self.pout, [0], [(PX_SUM, 1 + a, None) for a in range(len(self.aggs))],
                       max_groups=self.max_final, d_nrows=self.p_ng, key_range=rng, out=self.fout, ws=self.ws_f,
                       stream=stream, ngroups=self.f_ng,
                       flags=PX_AGG_STREAM if self.final_fresh else PX_AGG_ACCUMULATE)
        self.final_fresh = False
        self.partial_fresh = True
        self.emissions += 1
        self.events = [None, None]  # counts of the emitted Partial are stale

    def finish(self, stream=None) -> dict:
        self.emit(stream)
        return {"keys": self.fout[:1], "aggs": self.fout[1:], "ngroups": self.f_ng, "emissions": self.emissions}
