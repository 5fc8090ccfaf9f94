"""GPU parity of the fused join probe + aggregation (px_join_probe_agg): the
groups equal the oracle's join followed by group-by - per segment (Partial mode
after the exchange), unsegmented with a selection (Single mode), with probe keys
that miss, with group keys outside the statistic, and a multi-map table is
reported as unsupported."""
import numpy as np
import pytest
import torch

import oracle
import pxdata
from gpu_helpers import assert_groups_equal, count, dev, host

pytestmark = pytest.mark.gpu


def test_probe_agg_segmented_partial_matches_oracle(px):
    from paper_2606_24647_gb300.pipelines import AtScalePipeline
    d = pxdata.plain_at_scale(20_000, 400_000, nattr=500)
    want = oracle.pipeline_at_scale(d, 64)
    dd = {k: dev(v) for k, v in d.items()}
    p = AtScalePipeline(dd, nparts=64, nattr_bound=500, fused=True)
    r = p.run()
    assert p.ws.status() == px.PX_OK
    part = r["partial"]
    assert_groups_equal({"keys": part["keys"], "aggs": part["aggs"], "ngroups": part["ngroups"],
                         "seg": part["seg"]}, want["partial"], 1, segmented=True)
    assert_groups_equal(r["final"], want["final"], 1)
    # and the unfused pipeline gives the same final answer
    q = AtScalePipeline(dd, nparts=64, nattr_bound=500, fused=False).run()
    n = count(q["final"]["ngroups"])
    assert n == count(r["final"]["ngroups"])


@pytest.mark.parametrize("use_sel", [True, False])
@pytest.mark.parametrize("in_table", [False, True])
@pytest.mark.parametrize("rng", ["exact", "narrow"])
def test_probe_agg_single_with_selection_and_misses(px, rng, in_table, use_sel):
    # without a selection, SUM + COUNT runs through the lean probe-fed kernel
    d = pxdata.plain_join(20_000, 300_003, nattr=25)
    g = pxdata.rng(900)
    d["fk"][::11] = g.integers(20_001, 30_000, size=d["fk"][::11].size)  # keys with no match
    sel = oracle.filter(d["date"], pxdata.CFG2_DATE_LO, pxdata.CFG2_DATE_HI) if use_sel else None
    pr, br, _ = oracle.join(d["pk"], d["fk"], sel=sel)
    want = oracle.groupby([d["attr"][br]], [(oracle.SUM, d["amount"][pr], None), (oracle.COUNT, None, None)])
    dim = [dev(d["pk"]), dev(d["attr"])]
    # in_table: the group column is copied beside the keys and read from the table
    table = px.px_join_build(dim, 0, unique=True, pay_col=1 if in_table else None)
    lo, hi = (0, 24) if rng == "exact" else (5, 12)  # narrow: keys outside take the hash path
    kw = {"sel": dev(sel), "nsel": dev(np.array([sel.size], np.int64))} if use_sel else {}
    res = px.px_join_probe_agg(table, [dev(d["fk"]), dev(d["amount"])], 0, dim[1], (lo, hi),
                               [(px.PX_SUM, 1, None), (px.PX_COUNT, None, None)], max_groups=64, **kw)
    assert_groups_equal(res, want, 1)


def test_probe_agg_int8_group_copied_into_the_table(px):
    # a one-byte group column copied beside the keys (sign-extended like the gather)
    d = pxdata.plain_join(5_000, 200_001, nattr=25)
    g = pxdata.rng(901)
    grp = g.integers(-100, 100, size=d["pk"].size, dtype=np.int8)
    pr, br, _ = oracle.join(d["pk"], d["fk"])
    want = oracle.groupby([grp[br]], [(oracle.SUM, d["amount"][pr], None), (oracle.COUNT, None, None)])
    dim = [dev(d["pk"]), dev(grp)]
    for pay_col in (None, 1):
        table = px.px_join_build(dim, 0, unique=True, pay_col=pay_col)
        res = px.px_join_probe_agg(table, [dev(d["fk"]), dev(d["amount"])], 0, dim[1], (-100, 99),
                                   [(px.PX_SUM, 1, None), (px.PX_COUNT, None, None)], max_groups=256)
        assert_groups_equal(res, want, 1)


def test_probe_agg_multimap_table_is_unsupported(px):
    pk = np.array([1, 1, 2, 3], np.int64)
    attr = np.array([0, 1, 2, 3], np.int32)
    dim = [dev(pk), dev(attr)]
    table = px.px_join_build(dim, 0, unique=False)
    ws = px.Workspace(1 << 20)
    px.px_join_probe_agg(table, [dev(np.array([1, 2, 3], np.int64))], 0, dim[1], (0, 3),
                         [(px.PX_COUNT, None, None)], max_groups=8, ws=ws)
    assert ws.status() == px.PX_ERR_UNSUPPORTED
