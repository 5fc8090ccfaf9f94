"""GPU tests of the serving loop: every served query equals the CPU oracle's
fragment result, bit-exact, and the same whether it was served in a mix with
others (continuous batching), alone, or by the one-at-a-time server."""
import numpy as np
import pytest
import torch

import oracle
import pxdata
from gpu_helpers import count, dev, host

pytestmark = pytest.mark.gpu

LO, HI = pxdata.CFG2_DATE_LO, pxdata.CFG2_DATE_HI


def _setup(px, nq=40):
    from paper_2606_24647_gb300 import serving
    dims, dim_np = [], []
    for i, (nb, ng) in enumerate([(500, 5), (2000, 50), (20_000, 500), (100_000, 3000)]):
        d = pxdata.fragment(0, nb, ng, seed=500 + i)
        dims.append(serving.ResidentDim(dev(d["pk"]), dev(d["attr"]), ng))
        dim_np.append(d)
    g = pxdata.rng(77)
    queries, datas = [], []
    for q in range(nq):
        k = int(g.integers(0, len(dims)))
        nf = int(g.integers(1000, 50_000))
        d = pxdata.fragment(nf, dim_np[k]["pk"].size, dims[k].ngroups, seed=600 + q)
        d["pk"], d["attr"] = dim_np[k]["pk"], dim_np[k]["attr"]  # the resident dimension
        cols = {c: dev(d[c]) for c in ("key", "price", "qty", "date")}
        queries.append(serving.Query(q, dims[k], cols, LO, HI))
        datas.append(d)
    return serving, queries, datas


def _result(q):
    keys, aggs, ng = q.out
    n = count(ng)
    k = host(keys, n).astype(np.int64)
    o = np.argsort(k, kind="stable")
    return k[o], [host(a, n)[o] for a in aggs]


def test_served_queries_match_oracle_alone_and_mixed(px):
    serving, queries, datas = _setup(px)
    arr = serving.poisson_arrivals(4000.0, len(queries), seed=3)
    srv = serving.Server(budget_bytes=1 << 30, max_batch=16)
    stats = srv.serve(queries, arr)
    assert stats["queries"] == len(queries) and stats["p99_ms"] >= stats["p50_ms"] > 0
    mixed = [_result(q) for q in queries]
    for (k, aggs), d in zip(mixed, datas):
        want = oracle.pipeline_fragment(d, LO, HI)["groups"]
        np.testing.assert_array_equal(k, want["keys"][0])
        for a in range(3):
            np.testing.assert_array_equal(aggs[a], want["aggs"][a])
    # all at once (one big batch), then one at a time: identical results
    serving.Server(budget_bytes=1 << 30, max_batch=64).serve(queries, np.zeros(len(queries)))
    for (k, aggs), q in zip(mixed, queries):
        k2, aggs2 = _result(q)
        np.testing.assert_array_equal(k, k2)
        for a in range(3):
            np.testing.assert_array_equal(aggs[a], aggs2[a])
    serving.OneAtATimeServer().serve(queries, np.zeros(len(queries)))
    for (k, aggs), q in zip(mixed, queries):
        k2, aggs2 = _result(q)
        np.testing.assert_array_equal(k, k2)
        for a in range(3):
            np.testing.assert_array_equal(aggs[a], aggs2[a])


def test_budget_limits_what_is_in_flight(px):
    serving, queries, _ = _setup(px, nq=12)
    budget = max(q.nbytes for q in queries) + 10
    srv = serving.Server(budget_bytes=budget, max_batch=16)
    stats = srv.serve(queries, np.zeros(len(queries)))
    assert stats["peak_admitted_bytes"] <= budget
    assert stats["batches"] >= 6  # the budget forces small batches
