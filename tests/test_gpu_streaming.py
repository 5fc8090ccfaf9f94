"""GPU parity of streaming aggregation: Partial aggregation accumulating over a
stream of batches, emitting its groups into a Final stream past a size
threshold, must equal the oracle's Single aggregation over all rows - with the
dense key statistic, with keys outside it, and with no statistic (hash path)."""
import numpy as np
import pytest
import torch

import oracle
import pxdata
from gpu_helpers import count, dev, host

pytestmark = pytest.mark.gpu


def _stream(px, k, a, b, chunks, threshold, key_range, max_partial, max_final):
    from paper_2606_24647_gb300.pipelines import StreamingAggregation
    aggs = [(px.PX_SUM, 1, None), (px.PX_SUM_MUL, 1, 2), (px.PX_COUNT, None, None)]
    sa = StreamingAggregation(torch.int32, aggs, threshold=threshold, max_partial=max_partial, max_final=max_final,
                              key_range=key_range)
    n = k.size
    bounds = np.linspace(0, n, chunks + 1).astype(int)
    for i in range(chunks):
        lo, hi = bounds[i], bounds[i + 1]
        sa.feed([dev(k[lo:hi]), dev(a[lo:hi]), dev(b[lo:hi])], 0)
    r = sa.finish()
    torch.cuda.synchronize()
    assert sa.ws_p.status() == px.PX_OK and sa.ws_f.status() == px.PX_OK
    return r


@pytest.mark.parametrize("mode", ["dense", "outside", "hash"])
def test_streaming_partial_final_equals_single(px, mode):
    g = pxdata.rng(800)
    n = 600_000
    k = pxdata.random_column(g, n, np.int32, 0, 4999)
    if mode == "outside":
        k[::7] = 6000 + (np.arange(k[::7].size) % 300).astype(np.int32)  # outside the statistic
    a = pxdata.random_column(g, n, np.int64, -10**9, 10**9)
    b = pxdata.random_column(g, n, np.int64, 0, 100)
    want = oracle.groupby([k], [(oracle.SUM, a, None), (oracle.SUM_MUL, a, b), (oracle.COUNT, None, None)])
    kr = None if mode == "hash" else [(0, 4999)]
    r = _stream(px, k, a, b, chunks=24, threshold=1500, key_range=kr, max_partial=8192, max_final=8192)
    assert r["emissions"] >= 2
    ng = count(r["ngroups"])
    assert ng == want["ngroups"]
    keys = host(r["keys"][0], ng).astype(np.int64)
    o = np.argsort(keys)
    np.testing.assert_array_equal(keys[o], want["keys"][0])
    for i in range(3):
        np.testing.assert_array_equal(host(r["aggs"][i], ng)[o], want["aggs"][i])


def test_accumulate_over_calls_equals_one_call(px):
    g = pxdata.rng(801)
    n = 300_000
    k = pxdata.random_column(g, n, np.int32, -50, 50)
    a = pxdata.random_column(g, n, np.int64)
    one = px.px_groupby_agg([dev(k), dev(a)], [0], [(px.PX_SUM, 1, None), (px.PX_COUNT, None, None)],
                            max_groups=128, key_range=[(-50, 50)])
    ws = px.Workspace(1 << 20)
    out = [torch.empty(128, dtype=torch.int32, device="cuda")] + [torch.empty(128, dtype=torch.int64, device="cuda")
                                                                  for _ in range(2)]
    ng = torch.zeros(1, dtype=torch.int64, device="cuda")
    for i, (lo, hi) in enumerate([(0, 1000), (1000, 250_000), (250_000, n)]):
        res = px.px_groupby_agg([dev(k[lo:hi]), dev(a[lo:hi])], [0], [(px.PX_SUM, 1, None), (px.PX_COUNT, None, None)],
                                max_groups=128, key_range=[(-50, 50)], out=out, ws=ws, ngroups=ng,
                                flags=px.PX_AGG_STREAM if i == 0 else px.PX_AGG_ACCUMULATE)
    torch.cuda.synchronize()
    n1, n2 = count(one["ngroups"]), count(res["ngroups"])
    assert n1 == n2 == 101

    def canon(r, m):
        kk = host(r["keys"][0], m).astype(np.int64)
        o = np.argsort(kk)
        return kk[o], [host(x, m)[o] for x in r["aggs"]]
    k1, a1 = canon(one, n1)
    k2, a2 = canon(res, n2)
    np.testing.assert_array_equal(k1, k2)
    for x, y in zip(a1, a2):
        np.testing.assert_array_equal(x, y)
