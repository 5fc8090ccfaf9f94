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


def test_mix_with_at_scale_class_queries_under_a_binding_budget(px):
    """The served mix of the serving workload in small: fragment queries and, at
    about 1 in 10, at-scale-class queries (3M Zipf(1.1) keys over a 200k-row
    dimension: the fused kernel's large-fragment path), under a budget that fits
    one at-scale query but not two. Every query equals the oracle, and the same
    query gives the same result served in the mix and one at a time."""
    from paper_2606_24647_gb300 import serving
    big_np = pxdata.fragment(0, 200_000, 7_000, seed=700)
    small_np = pxdata.fragment(0, 20_000, 300, seed=701)
    big = serving.ResidentDim(dev(big_np["pk"]), dev(big_np["attr"]), 7_000)
    small = serving.ResidentDim(dev(small_np["pk"]), dev(small_np["attr"]), 300)
    g = pxdata.rng(78)
    queries, datas = [], []
    for q in range(22):
        if q % 10 == 3:  # at-scale class
            gg = pxdata.rng(710 + q)
            pk_of_rank = gg.permutation(big_np["pk"])
            key = pk_of_rank[pxdata.zipf_ranks(gg, pk_of_rank.size, 3_000_000, 1.1) - 1]
            d = pxdata.fragment(key.size, 1, 1, seed=720 + q)
            d["key"] = key
            dim, dnp = big, big_np
        else:
            d = pxdata.fragment(int(g.integers(1000, 80_000)), small_np["pk"].size, 300, seed=740 + q)
            dim, dnp = small, small_np
        d["pk"], d["attr"] = dnp["pk"], dnp["attr"]
        queries.append(serving.Query(q, dim, {c: dev(d[c]) for c in ("key", "price", "qty", "date")}, LO, HI))
        datas.append(d)
    nbig = max(q.nbytes for q in queries)
    budget = nbig + 4 * max(q.nbytes for q, d in zip(queries, datas) if d["key"].size < 1_000_000)
    assert budget < 2 * nbig  # two at-scale queries never fit together
    stats = serving.Server(budget_bytes=budget, max_batch=16).serve(
        queries, serving.poisson_arrivals(2000.0, len(queries), seed=9))
    assert stats["peak_admitted_bytes"] <= budget
    mixed = [_result(q) for q in queries]
    for (k, aggs), d in zip(mixed, datas):
        want = oracle.pipeline_fragment(d, LO, HI)["groups"]
        np.testing.assert_array_equal(k, want["keys"][0])
        for a in range(3):
            np.testing.assert_array_equal(aggs[a], want["aggs"][a])
    serving.OneAtATimeServer().serve(queries, np.zeros(len(queries)))
    for (k, aggs), q in zip(mixed, queries):
        k2, aggs2 = _result(q)
        np.testing.assert_array_equal(k, k2)
        for a in range(3):
            np.testing.assert_array_equal(aggs[a], aggs2[a])
