"""GPU parity of the batched fused fragments (px_fragments_run) against the CPU
oracle's fragment pipeline (filter -> join -> group-by), fragment by fragment,
bit-exact: the fused kernel's output is in ascending group-key order, like the
oracle's. Covers both aggregation modes (block arrays in shared memory, and
reductions straight into the global arrays), fragments without COUNT, empty and
one-group fragments, missing keys, every launch configuration (results must not
depend on it), and a group key outside the declared range."""
import numpy as np
import pytest
import torch

import oracle
import pxdata
from gpu_helpers import count, dev, host

pytestmark = pytest.mark.gpu

LO, HI = pxdata.CFG2_DATE_LO, pxdata.CFG2_DATE_HI


def _frag(px, d, ngroups, aggs=None, filtered=True):
    dim = [dev(d["pk"]), dev(d["attr"])]
    table = torch.empty(px.load().px_join_table_bytes(max(1, d["pk"].size), 0), dtype=torch.uint8, device="cuda")
    px.px_join_build(dim, 0, unique=True, table=table)
    f = {"key": dev(d["key"]), "cols": [dev(d["price"]), dev(d["qty"])],
         "aggs": aggs if aggs is not None else [(px.PX_SUM, 0, None), (px.PX_SUM_MUL, 0, 1), (px.PX_COUNT, None, None)],
         "table": table, "group": dim[1], "group_lo": 0, "group_hi": ngroups - 1, "max_groups": ngroups,
         "_dim": dim}
    if filtered:
        f.update(filter=dev(d["date"]), lo=LO, hi=HI)
    return f


def _want(d, filtered=True, ops=None):
    if filtered:
        return oracle.pipeline_fragment(d, LO, HI)["groups"]
    return oracle.pipeline_fragment(d, -(2**31), 2**31 - 1)["groups"]


def _check(res, want, naggs=3, which=None):
    n = count(res["ngroups"])
    assert n == want["ngroups"]
    np.testing.assert_array_equal(host(res["keys"], n).astype(np.int64), want["keys"][0])
    idx = which if which is not None else list(range(naggs))
    for a, w in enumerate(idx):
        np.testing.assert_array_equal(host(res["aggs"][a], n), want["aggs"][w])


def _mixed_batch(px, nfrags=24, seed=40):
    sz = pxdata.fragment_sizes(nfrags, seed=seed, scale=0.01)
    datas, frags = [], []
    for i in range(nfrags):
        d = pxdata.fragment(int(sz["nfact"][i]), int(sz["nbuild"][i]), int(sz["ngroups"][i]), seed=1000 + i)
        datas.append(d)
        frags.append(_frag(px, d, int(sz["ngroups"][i])))
    # edge cases: empty fact, one group, large shared-mode fragment, direct-mode fragment
    extra = [(0, 50, 7), (3000, 40, 1), (300_000, 2000, 60), (5000, 20_000, 20_000), (1, 1, 3)]
    for j, (nf, nb, ng) in enumerate(extra):
        d = pxdata.fragment(nf, nb, ng, seed=2000 + j)
        datas.append(d)
        frags.append(_frag(px, d, ng))
    return datas, frags


def test_fragments_parity_mixed_batch(px):
    datas, frags = _mixed_batch(px)
    fb = px.FragmentBatch(frags)
    res = fb.run()
    torch.cuda.synchronize()
    assert fb.ws.status() == px.PX_OK
    for d, r in zip(datas, res):
        _check(r, _want(d))


@pytest.mark.parametrize("cfg", [(256, 2, 512, 8), (256, 4, 2048, 2), (512, 2, 4096, 1), (512, 4, 65536, 2)])
def test_fragments_results_do_not_depend_on_config(px, cfg):
    datas, frags = _mixed_batch(px, nfrags=12, seed=41)
    fb = px.FragmentBatch(frags, config=cfg)
    res = fb.run()
    torch.cuda.synchronize()
    assert fb.ws.status() == px.PX_OK
    for d, r in zip(datas, res):
        _check(r, _want(d))
    # run again on the same batch: identical
    res2 = fb.run()
    torch.cuda.synchronize()
    for d, r in zip(datas, res2):
        _check(r, _want(d))


def test_fragments_alone_equals_in_batch(px):
    datas, frags = _mixed_batch(px, nfrags=10, seed=42)
    batch = px.FragmentBatch(frags).run()
    torch.cuda.synchronize()
    for i in [0, 3, 7, len(frags) - 2]:
        alone = px.FragmentBatch([frags[i]]).run()[0]
        torch.cuda.synchronize()
        n = count(alone["ngroups"])
        assert n == count(batch[i]["ngroups"])
        np.testing.assert_array_equal(host(alone["keys"], n), host(batch[i]["keys"], n))
        for a in range(3):
            np.testing.assert_array_equal(host(alone["aggs"][a], n), host(batch[i]["aggs"][a], n))


def test_fragments_without_count_and_without_filter(px):
    # occupancy flags decide which groups exist; a zero sum still makes a group
    d1 = pxdata.fragment(200_000, 3000, 40, seed=3001)     # shared mode
    d2 = pxdata.fragment(4000, 30_000, 30_000, seed=3002)  # direct mode
    d3 = pxdata.fragment(50_000, 500, 16, seed=3003)
    d3["price"][:] = 0                                     # all sums zero: groups still exist
    frags = [_frag(px, d1, 40, aggs=[(px.PX_SUM, 0, None)]),
             _frag(px, d2, 30_000, aggs=[(px.PX_SUM_MUL, 0, 1)], filtered=False),
             _frag(px, d3, 16, aggs=[(px.PX_SUM, 0, None)])]
    res = px.FragmentBatch(frags).run()
    torch.cuda.synchronize()
    _check(res[0], _want(d1), which=[0])
    _check(res[1], _want(d2, filtered=False), which=[1])
    _check(res[2], _want(d3), which=[0])


def test_fragments_group_key_outside_range_is_reported(px):
    d = pxdata.fragment(20_000, 1000, 50, seed=3004)
    f = _frag(px, d, 50)
    f["group_hi"] = 9  # keys go up to 49
    fb = px.FragmentBatch([f])
    fb.run()
    assert fb.ws.status() == px.PX_ERR_UNSUPPORTED


def test_fragments_capacity_overflow_is_reported(px):
    d = pxdata.fragment(20_000, 1000, 50, seed=3005)
    f = _frag(px, d, 50)
    f["max_groups"] = 10
    fb = px.FragmentBatch([f])
    r = fb.run()[0]
    assert fb.ws.status() == px.PX_ERR_CAPACITY
    want = _want(d)
    assert count(r["ngroups"]) == want["ngroups"]
    np.testing.assert_array_equal(host(r["keys"], 10).astype(np.int64), want["keys"][0][:10])


def test_fragments_bad_arguments_are_rejected(px):
    d = pxdata.fragment(100, 10, 4, seed=3006)
    f = _frag(px, d, 4)
    f["group_hi"] = 1 << 23  # over PX_FRAG_MAX_GROUPS
    with pytest.raises(px.PxError):
        px.FragmentBatch([f]).run()
    f = _frag(px, d, 4)
    with pytest.raises(px.PxError):
        px.FragmentBatch([f], config=(128, 4, 512, 1)).run()
