"""GPU parity of each operator against the CPU oracle, element by element, on
seeded inputs that span many tiles, ragged tails and the edge cases (empty
inputs, one row, all rows in one partition, duplicate keys, wrap-around sums,
capacity overflow). All integer work: the bar is bit-exact."""
import numpy as np
import pytest
import torch

import oracle
import pxdata
from gpu_helpers import assert_groups_equal, count, dev, host

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 31, 2047, 2048, 2049, 4095, 4096, 4097, 100_003]


# -------------------------------------------------------------- filter -----

@pytest.mark.parametrize("dtype", [np.int8, np.int32, np.int64])
def test_filter_parity(px, dtype):
    g = pxdata.rng(100)
    info = np.iinfo(dtype)
    for n in SIZES:
        col = pxdata.random_column(g, n, dtype)
        for lo, hi in [(info.min, info.max), (-10, 10**6), (0, 0), (int(info.max), int(info.min)),
                       (-(2**63), 2**63 - 1)]:
            sel, nsel = px.px_filter(dev(col), lo, hi)
            want = oracle.filter(col, lo, hi)
            assert count(nsel) == want.size
            np.testing.assert_array_equal(host(sel, want.size), want)


def test_filter_device_row_count(px):
    g = pxdata.rng(101)
    col = pxdata.random_column(g, 50_000, np.int32, 0, 2556)
    for n in [0, 1, 12_345, 50_000]:
        d_n = dev(np.array([n], np.int64))
        sel, nsel = px.px_filter(dev(col), 100, 2000, d_nrows=d_n)
        want = oracle.filter(col[:n], 100, 2000)
        assert count(nsel) == want.size
        np.testing.assert_array_equal(host(sel, want.size), want)


def test_filter_tile_counts_scanned_in_several_rounds(px):
    # More than 8192 tiles of 2048 rows: the one-block scan of the tile counts
    # carries its total across rounds; a ragged last tile and a d_nrows cut too.
    g = pxdata.rng(102)
    n = 8192 * 2048 * 2 + 12_345
    col = pxdata.random_column(g, n, np.int8)
    for lo, hi, cut in [(-20, 90, n), (0, 1, n - 777)]:
        d_n = dev(np.array([cut], np.int64))
        sel, nsel = px.px_filter(dev(col), lo, hi, d_nrows=d_n)
        want = oracle.filter(col[:cut], lo, hi)
        assert count(nsel) == want.size
        np.testing.assert_array_equal(host(sel, want.size), want)


# ----------------------------------------------------------- partition -----

def _part_cols(g, n):
    return [pxdata.random_column(g, n, np.int64, -(2**40), 2**40),
            pxdata.random_column(g, n, np.int32),
            pxdata.random_column(g, n, np.int8),
            np.arange(n, dtype=np.int64)]


@pytest.mark.parametrize("P", [1, 2, 3, 8, 64, 1000, 1024])
def test_partition_parity(px, P):
    g = pxdata.rng(200 + P)
    for n in [0, 1, 4095, 4096, 4097, 60_001]:
        cols = _part_cols(g, n)
        for seed in [0, 0xDEADBEEF12345678]:
            out, off = px.px_partition([dev(c) for c in cols], 0, P, seed)
            want, woff = oracle.partition(cols, 0, P, seed)
            np.testing.assert_array_equal(host(off), woff)
            for a, b in zip(out, want):
                np.testing.assert_array_equal(host(a, n), b)


@pytest.mark.parametrize("P", [3, 64, 1000])
def test_partition_parity_long_count_rows(px, P):
    # a count matrix of more than 4096 tiles per partition (several scan tiles per row)
    g = pxdata.rng(220 + P)
    n = 8_400_777
    cols = _part_cols(g, n)
    for d_n in [None, 8_390_001]:
        kw = {} if d_n is None else {"d_nrows": dev(np.array([d_n], np.int64))}
        m = n if d_n is None else d_n
        out, off = px.px_partition([dev(c) for c in cols], 0, P, 5, **kw)
        want, woff = oracle.partition([c[:m] for c in cols], 0, P, 5)
        np.testing.assert_array_equal(host(off), woff)
        for a, b in zip(out, want):
            np.testing.assert_array_equal(host(a, m), b)


def test_partition_with_selection_and_key_not_first(px):
    g = pxdata.rng(210)
    n = 70_001
    cols = _part_cols(g, n)
    cols = [cols[1], cols[0], cols[2], cols[3]]
    sel = oracle.filter(cols[1], -(2**39), 2**39)
    out, off = px.px_partition([dev(c) for c in cols], 1, 64, 7, sel=dev(sel), nsel=dev(np.array([sel.size])))
    want, woff = oracle.partition(cols, 1, 64, 7, sel=sel)
    np.testing.assert_array_equal(host(off), woff)
    for a, b in zip(out, want):
        np.testing.assert_array_equal(host(a, sel.size), b)


def test_partition_skew_all_one_key(px):
    n = 50_000
    key = np.full(n, 42, np.int64)
    rid = np.arange(n, dtype=np.int32)
    out, off = px.px_partition([dev(key), dev(rid)], 0, 64, 0)
    want, woff = oracle.partition([key, rid], 0, 64, 0)
    np.testing.assert_array_equal(host(off), woff)
    np.testing.assert_array_equal(host(out[1], n), want[1])


def test_partition_device_row_count(px):
    g = pxdata.rng(211)
    cols = _part_cols(g, 30_000)
    for n in [0, 5, 9_999]:
        out, off = px.px_partition([dev(c) for c in cols], 0, 8, 0, d_nrows=dev(np.array([n], np.int64)))
        want, woff = oracle.partition([c[:n] for c in cols], 0, 8, 0)
        np.testing.assert_array_equal(host(off), woff)
        for a, b in zip(out, want):
            np.testing.assert_array_equal(host(a, n), b)


# ---------------------------------------------------------------- join -----

def _join(px, pk, fk, unique=True, sel=None, bseg=None, pseg=None, out_cap=None, payload_dtype=np.int32):
    g = pxdata.rng(300)
    attr = pxdata.random_column(g, pk.size, payload_dtype)
    amount = pxdata.random_column(g, fk.size, np.int64)
    ws = px.Workspace(1 << 20)
    table = px.px_join_build([dev(pk)], 0, seg=None if bseg is None else dev(bseg), unique=unique, ws=ws)
    kw = {}
    if sel is not None:
        kw = {"sel": dev(sel), "nsel": dev(np.array([sel.size], np.int64))}
    res = px.px_join_probe(table, [dev(fk), dev(amount)], 0, carry=[1], payload=[dev(attr)],
                           seg=None if pseg is None else dev(pseg), probe_row=True, build_row=True,
                           out_seg=pseg is not None, out_cap=out_cap, ws=ws, **kw)
    return res, attr, amount, ws


def test_join_unique_parity(px):
    g = pxdata.rng(301)
    for nb, nprobe in [(0, 100), (100, 0), (1, 1), (1000, 5000), (20_000, 100_003)]:
        pk = (g.permutation(3 * max(nb, 1))[:nb] - nb).astype(np.int64)
        fk = pxdata.random_column(g, nprobe, np.int64, -nb, 2 * nb)
        for sel in [None, oracle.filter(pxdata.random_column(g, nprobe, np.int32, 0, 9), 0, 3)]:
            res, attr, amount, ws = _join(px, pk, fk, sel=sel)
            assert ws.status() == px.PX_OK
            pr, br, _ = oracle.join(pk, fk, sel=sel)
            m = count(res["nout"])
            assert m == pr.size
            np.testing.assert_array_equal(host(res["probe_row"], m), pr)
            np.testing.assert_array_equal(host(res["build_row"], m), br)
            np.testing.assert_array_equal(host(res["cols"][0], m), amount[pr])
            np.testing.assert_array_equal(host(res["cols"][1], m), attr[br])


def test_join_full_tiles_next_to_partial_tiles(px):
    # every position of the first tiles matches (ranked without ballots), then
    # tiles with misses, then a selection that makes every tile partial again
    g = pxdata.rng(309)
    pk = g.permutation(50_000).astype(np.int64)
    fk = np.concatenate([pk[g.integers(0, pk.size, 40_960)],
                         pxdata.random_column(g, 30_001, np.int64, -20_000, 70_000),
                         pk[g.integers(0, pk.size, 5_000)]])
    for sel in [None, oracle.filter(pxdata.random_column(g, fk.size, np.int32, 0, 9), 0, 7)]:
        res, attr, amount, ws = _join(px, pk, fk, sel=sel)
        assert ws.status() == px.PX_OK
        pr, br, _ = oracle.join(pk, fk, sel=sel)
        m = count(res["nout"])
        assert m == pr.size
        np.testing.assert_array_equal(host(res["probe_row"], m), pr)
        np.testing.assert_array_equal(host(res["build_row"], m), br)
        np.testing.assert_array_equal(host(res["cols"][0], m), amount[pr])
        np.testing.assert_array_equal(host(res["cols"][1], m), attr[br])


def test_join_table_at_a_16_byte_offset(px):
    # the table is caller memory aligned to 16 bytes only; its buckets are padded
    # to 64-byte addresses inside it
    g = pxdata.rng(310)
    pk = g.permutation(30_000).astype(np.int64)
    fk = pxdata.random_column(g, 70_000, np.int64, -1000, 31_000)
    L = px.load()
    need = L.px_join_table_bytes(pk.size, 0)
    buf = torch.empty(need + 64, dtype=torch.uint8, device="cuda")
    pr, br, _ = oracle.join(pk, fk)
    for off in (16, 32, 48):
        table = buf[off:off + need]
        ws = px.Workspace(1 << 20)
        px.px_join_build([dev(pk)], 0, table=table, ws=ws)
        res = px.px_join_probe(table, [dev(fk)], 0, probe_row=True, build_row=True, ws=ws)
        assert ws.status() == px.PX_OK
        m = count(res["nout"])
        assert m == pr.size
        np.testing.assert_array_equal(host(res["probe_row"], m), pr)
        np.testing.assert_array_equal(host(res["build_row"], m), br)


@pytest.mark.parametrize("nb", [65_534, 65_535, 70_000])
def test_join_around_two_to_the_16_build_rows(px, nb):
    # unique tables of about 2^16 build rows, whole and cut into segments, with
    # probes that mostly match and a tail of misses
    g = pxdata.rng(311)
    pk = (g.permutation(nb) * 3 + 1).astype(np.int64)
    fk = np.concatenate([pk[g.integers(0, nb, 90_000)], pxdata.random_column(g, 20_001, np.int64, 0, 3 * nb)])
    for seg in [None, np.array([0, 1000, nb // 2, nb], np.int64)]:
        pseg = None if seg is None else np.array([0, 10_000, 60_000, fk.size], np.int64)
        res, attr, amount, ws = _join(px, pk, fk, bseg=seg, pseg=pseg)
        assert ws.status() == px.PX_OK
        pr, br, oseg = oracle.join(pk, fk, build_seg=seg, probe_seg=pseg)
        m = count(res["nout"])
        assert m == pr.size
        np.testing.assert_array_equal(host(res["probe_row"], m), pr)
        np.testing.assert_array_equal(host(res["build_row"], m), br)
        np.testing.assert_array_equal(host(res["cols"][1], m), attr[br])
        if pseg is not None:
            np.testing.assert_array_equal(host(res["out_seg"]), oseg)


def test_join_multi_match_parity(px):
    g = pxdata.rng(302)
    pk = pxdata.random_column(g, 3000, np.int64, 0, 700)       # ~4 duplicates per key
    fk = pxdata.random_column(g, 20_000, np.int64, -50, 750)
    pr, br, _ = oracle.join(pk, fk)
    res, attr, amount, ws = _join(px, pk, fk, unique=False, out_cap=pr.size)
    assert ws.status() == px.PX_OK
    m = count(res["nout"])
    assert m == pr.size
    gpr, gbr = host(res["probe_row"], m), host(res["build_row"], m)
    np.testing.assert_array_equal(gpr, pr)            # probe order is unique
    # the matches of one probe row may come in any order: compare per-row multisets
    order_g = np.lexsort((gbr, gpr))
    np.testing.assert_array_equal(gbr[order_g], br)
    np.testing.assert_array_equal(host(res["cols"][0], m), amount[gpr])
    np.testing.assert_array_equal(host(res["cols"][1], m), attr[gbr])


def test_join_segmented_parity(px):
    g = pxdata.rng(303)
    d = pxdata.plain_at_scale(20_000, 300_000, nattr=50)
    dparts, doff = oracle.partition([d["pk"]], 0, 64, 0)
    fparts, foff = oracle.partition([d["fk"]], 0, 64, 0)
    res, attr, amount, ws = _join(px, dparts[0], fparts[0], bseg=doff, pseg=foff)
    assert ws.status() == px.PX_OK
    pr, br, oseg = oracle.join(dparts[0], fparts[0], build_seg=doff, probe_seg=foff)
    m = count(res["nout"])
    assert m == pr.size == 300_000
    np.testing.assert_array_equal(host(res["probe_row"], m), pr)
    np.testing.assert_array_equal(host(res["build_row"], m), br)
    np.testing.assert_array_equal(host(res["out_seg"]), oseg)


def test_join_segments_with_empty_segments(px):
    g = pxdata.rng(304)
    pk = pxdata.random_column(g, 500, np.int64, 0, 300)
    pk = np.unique(pk)
    fk = pxdata.random_column(g, 4000, np.int64, 0, 300)
    bseg = np.array([0, 0, pk.size // 3, pk.size // 3, pk.size, pk.size], np.int64)
    pseg = np.array([0, 100, 100, 2500, 4000, 4000], np.int64)
    res, attr, amount, ws = _join(px, pk, fk, bseg=bseg, pseg=pseg)
    assert ws.status() == px.PX_OK
    pr, br, oseg = oracle.join(pk, fk, build_seg=bseg, probe_seg=pseg)
    m = count(res["nout"])
    assert m == pr.size
    np.testing.assert_array_equal(host(res["probe_row"], m), pr)
    np.testing.assert_array_equal(host(res["build_row"], m), br)
    np.testing.assert_array_equal(host(res["out_seg"]), oseg)


def test_join_duplicate_key_is_reported(px):
    pk = np.array([5, 6, 7, 6], np.int64)
    ws = px.Workspace(1 << 16)
    px.px_join_build([dev(pk)], 0, unique=True, ws=ws)
    assert ws.status() == px.PX_ERR_DUPLICATE_KEY


def test_join_reserved_key_is_reported(px):
    pk = np.array([5, -(2**63), 7], np.int64)
    ws = px.Workspace(1 << 16)
    px.px_join_build([dev(pk)], 0, unique=True, ws=ws)
    assert ws.status() == px.PX_ERR_UNSUPPORTED


def test_join_capacity_overflow_reports_required_size(px):
    pk = np.arange(100, dtype=np.int64)
    fk = np.tile(np.arange(100, dtype=np.int64), 30)
    res, attr, amount, ws = _join(px, pk, fk, out_cap=1000)
    assert ws.status() == px.PX_ERR_CAPACITY
    assert count(res["nout"]) == 3000
    pr, br, _ = oracle.join(pk, fk)
    np.testing.assert_array_equal(host(res["probe_row"], 1000), pr[:1000])


# ------------------------------------------------------------ group-by -----

def _gb(px, cols, key_idx, aggs, max_groups, **kw):
    return px.px_groupby_agg([dev(c) for c in cols], key_idx, aggs, max_groups=max_groups, **kw)


@pytest.mark.parametrize("kt", [(np.int8,), (np.int32,), (np.int64,), (np.int8, np.int8), (np.int32, np.int8),
                                (np.int32, np.int32)])
def test_groupby_parity(px, kt):
    g = pxdata.rng(400)
    for n in [0, 1, 2047, 2049, 100_003]:
        for dom in [3, 300, 30_000]:
            keys = [pxdata.random_column(g, n, t, max(np.iinfo(t).min, -dom), min(np.iinfo(t).max, dom))
                    for t in kt]
            a64 = pxdata.random_column(g, n, np.int64)
            a32 = pxdata.random_column(g, n, np.int32)
            b8 = pxdata.random_column(g, n, np.int8)
            cols = keys + [a64, a32, b8]
            nk = len(kt)
            aggs = [(px.PX_SUM, nk, None), (px.PX_COUNT, None, None), (px.PX_SUM_MUL, nk + 1, nk + 2),
                    (px.PX_SUM_MUL, nk, nk)]
            want = oracle.groupby(keys, [(oracle.SUM, a64, None), (oracle.COUNT, None, None),
                                         (oracle.SUM_MUL, a32, b8), (oracle.SUM_MUL, a64, a64)])
            # hash path (no statistic), exact range, half range (dense + spill), wrong range
            for rng in [None, "exact", "half", "wrong"]:
                kr = None
                if rng is not None and n:
                    lo = [int(k.min()) for k in keys]
                    hi = [int(k.max()) for k in keys]
                    if rng == "half":
                        hi = [l + (h - l) // 2 for l, h in zip(lo, hi)]
                    elif rng == "wrong":
                        lo, hi = [h + 1 for h in hi], [h + 5 for h in hi]
                    kr = list(zip(lo, hi))
                res = _gb(px, cols, list(range(nk)), aggs, max(1, want["ngroups"]), key_range=kr)
                assert_groups_equal(res, want, nk)


def test_groupby_selection_and_device_count(px):
    g = pxdata.rng(401)
    n = 80_000
    k = pxdata.random_column(g, n, np.int32, 0, 99)
    a = pxdata.random_column(g, n, np.int64, -10**9, 10**9)
    sel = oracle.filter(pxdata.random_column(g, n, np.int32, 0, 9), 0, 4)
    want = oracle.groupby([k], [(oracle.SUM, a, None), (oracle.COUNT, None, None)], sel=sel)
    res = _gb(px, [k, a], [0], [(px.PX_SUM, 1, None), (px.PX_COUNT, None, None)], 128, sel=dev(sel),
              nsel=dev(np.array([sel.size], np.int64)))
    assert_groups_equal(res, want, 1)
    want = oracle.groupby([k[:5000]], [(oracle.SUM, a[:5000], None), (oracle.COUNT, None, None)])
    res = _gb(px, [k, a], [0], [(px.PX_SUM, 1, None), (px.PX_COUNT, None, None)], 128,
              d_nrows=dev(np.array([5000], np.int64)))
    assert_groups_equal(res, want, 1)


def test_groupby_segmented_parity(px):
    g = pxdata.rng(402)
    n = 120_000
    k = pxdata.random_column(g, n, np.int32, 0, 2000)
    a = pxdata.random_column(g, n, np.int64, 0, 10**6)
    seg = np.array([0, 0, 100, 101, 60_000, 60_000, 119_999, n], np.int64)
    want = oracle.groupby([k], [(oracle.SUM, a, None), (oracle.COUNT, None, None)], seg=seg)
    res = _gb(px, [k, a], [0], [(px.PX_SUM, 1, None), (px.PX_COUNT, None, None)], want["ngroups"], seg=dev(seg))
    assert_groups_equal(res, want, 1, segmented=True)


def test_groupby_hot_key_and_wrap(px):
    n = 200_000
    k = np.zeros(n, np.int8)
    k[::1000] = 1
    a = np.full(n, 2**62 + 12345, np.int64)   # sums wrap mod 2^64
    want = oracle.groupby([k], [(oracle.SUM, a, None), (oracle.SUM_MUL, a, a), (oracle.COUNT, None, None)])
    res = _gb(px, [k, a], [0], [(px.PX_SUM, 1, None), (px.PX_SUM_MUL, 1, 1), (px.PX_COUNT, None, None)], 4)
    assert_groups_equal(res, want, 1)


def test_groupby_many_groups_spill_to_global(px):
    g = pxdata.rng(403)
    n = 300_000
    k = pxdata.random_column(g, n, np.int64, -(2**62), 2**62)   # ~all distinct
    k[::3] = 77                                                 # plus one hot key
    a = pxdata.random_column(g, n, np.int64, 0, 1000)
    want = oracle.groupby([k], [(oracle.SUM, a, None), (oracle.COUNT, None, None)])
    res = _gb(px, [k, a], [0], [(px.PX_SUM, 1, None), (px.PX_COUNT, None, None)], want["ngroups"])
    assert_groups_equal(res, want, 1)


@pytest.mark.parametrize("dense", [False, True])
def test_groupby_without_count_distinct_and_many_aggs(px, dense):
    g = pxdata.rng(404)
    n = 150_001
    k0 = pxdata.random_column(g, n, np.int32, -20, 20)
    k1 = pxdata.random_column(g, n, np.int8, 0, 3)
    a = pxdata.random_column(g, n, np.int64, -10**12, 10**12)
    b = pxdata.random_column(g, n, np.int32)
    kr = [(-20, 20), (0, 3)] if dense else None
    cols = [k0, k1, a, b]
    # no COUNT: occupancy comes from a bitmap in dense mode
    want = oracle.groupby([k0, k1], [(oracle.SUM, a, None), (oracle.SUM_MUL, a, b)])
    res = _gb(px, cols, [0, 1], [(px.PX_SUM, 2, None), (px.PX_SUM_MUL, 2, 3)], want["ngroups"], key_range=kr)
    assert_groups_equal(res, want, 2)
    # DISTINCT: no aggregates at all
    want = oracle.groupby([k0, k1], [])
    res = _gb(px, cols, [0, 1], [], want["ngroups"], key_range=kr)
    assert_groups_equal(res, want, 2)
    # more than four aggregates (the generic kernel)
    ops = [(oracle.SUM, a, None), (oracle.COUNT, None, None), (oracle.SUM, b, None), (oracle.SUM_MUL, a, b),
           (oracle.SUM_MUL, b, b), (oracle.SUM, k0, None)]
    gops = [(px.PX_SUM, 2, None), (px.PX_COUNT, None, None), (px.PX_SUM, 3, None), (px.PX_SUM_MUL, 2, 3),
            (px.PX_SUM_MUL, 3, 3), (px.PX_SUM, 0, None)]
    want = oracle.groupby([k0, k1], ops)
    res = _gb(px, cols, [0, 1], gops, want["ngroups"], key_range=kr)
    assert_groups_equal(res, want, 2)


def test_groupby_dense_segmented_hot_partition(px):
    # Partial mode over Zipf-skewed segments with the dense path (the at-scale shape).
    d = pxdata.plain_at_scale(20_000, 400_000, nattr=500)
    pr, br, _ = oracle.join(d["pk"], d["fk"])
    attr, amount = d["attr"][br], d["amount"][pr]
    seg = np.array([0, 1000, 1000, 250_000, 399_999, 400_000], np.int64)
    want = oracle.groupby([attr], [(oracle.SUM, amount, None), (oracle.COUNT, None, None)], seg=seg)
    res = _gb(px, [attr, amount], [0], [(px.PX_SUM, 1, None), (px.PX_COUNT, None, None)], want["ngroups"],
              seg=dev(seg), key_range=[(0, 499)])
    assert_groups_equal(res, want, 1, segmented=True)


@pytest.mark.parametrize("n", [200_000, 1_500_000])
def test_groupby_dense_global_direct_and_block(px, n):
    # max_groups covers the whole (segment, key) space, so results go to the dense
    # global array: 200K rows add into it row by row (too few rows to give each of
    # the 152 SMs a block that amortises its block arrays); 1.5M rows use block
    # arrays flushed per segment. Zipf-skewed keys from the at-scale shape.
    d = pxdata.plain_at_scale(20_000, n, nattr=700)
    pr, br, _ = oracle.join(d["pk"], d["fk"])
    attr, amount = d["attr"][br], d["amount"][pr]
    seg = np.array([0, n // 7, n // 7, n // 2, n - 3, n], np.int64)
    want = oracle.groupby([attr], [(oracle.SUM, amount, None), (oracle.COUNT, None, None)], seg=seg)
    res = _gb(px, [attr, amount], [0], [(px.PX_SUM, 1, None), (px.PX_COUNT, None, None)], 5 * 700,
              seg=dev(seg), key_range=[(0, 699)])
    assert_groups_equal(res, want, 1, segmented=True)
    # without COUNT (occupancy bitmap) and a key outside the range (global path)
    attr2 = attr.copy()
    attr2[::9973] = 5000
    want = oracle.groupby([attr2], [(oracle.SUM, amount, None)], seg=seg)
    res = _gb(px, [attr2, amount], [0], [(px.PX_SUM, 1, None)], 5 * 700 + 64, seg=dev(seg),
              key_range=[(0, 699)])
    assert_groups_equal(res, want, 1, segmented=True)


def test_groupby_capacity_overflow_reported(px):
    k = np.arange(1000, dtype=np.int32)
    ws = px.Workspace(1 << 20)
    res = px.px_groupby_agg([dev(k)], [0], [(px.PX_COUNT, None, None)], max_groups=100, ws=ws)
    assert ws.status() == px.PX_ERR_CAPACITY
    assert count(res["ngroups"]) == 1000


# ------------------------------------------------------- bounded waits -----

def test_bounded_wait_times_out_and_context_stays_usable(px):
    # a flag nothing sets: the device wait gives up with PX_ERR_TIMEOUT (no hang,
    # no fault), and the context keeps working afterwards
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    px.px_selftest_wait(flag, 20_000, status)
    assert count(status) == px.PX_ERR_TIMEOUT
    flag.fill_(1)
    px.px_selftest_wait(flag, 20_000, status)
    assert count(status) == px.PX_OK
    col = dev(np.arange(1000, dtype=np.int32))
    sel, nsel = px.px_filter(col, 10, 20)
    assert count(nsel) == 10
    with pytest.raises(px.PxError):
        px.px_selftest_wait(flag, 0, status)


def test_partition_every_launch_shape_gives_the_same_result(px):
    """Every point of the autotuner's exchange grid: identical offsets and columns
    (equal to the oracle's), on a skewed input spanning many tiles per block."""
    from paper_2606_24647_gb300 import autotune
    d = pxdata.plain_at_scale(20_000, 700_001, nattr=100, seed=31)
    cols_np = [d["fk"], d["amount"], d["date"]]
    cols = [dev(c) for c in cols_np]
    want, woff = oracle.partition(cols_np, 0, 64, 0)
    for cfg in autotune.PARTITION_GRID + [(0, 0)]:
        out, off = px.px_partition(cols, 0, 64, 0, config=cfg)
        np.testing.assert_array_equal(host(off), woff)
        for c in range(3):
            np.testing.assert_array_equal(host(out[c]), want[c])


@pytest.mark.parametrize("kt,vt", [(np.int32, np.int64), (np.int32, np.int32), (np.int64, np.int64),
                                   (np.int64, np.int32)])
def test_groupby_sum_count_wide_key_range(px, kt, vt):
    """SUM + COUNT over a key range of 8193..16384 slots with a dense global result
    and enough rows for dense block aggregation: the shape the lean sum-count kernel
    serves (one shared-memory replica per block; the smaller input takes the direct
    mode). Zipf-skewed keys (hot-key warp sums), keys outside the statistic (global
    path), full-range values (carries into the high word, negatives), segments with
    empty ones and boundaries off the tile grid, a ragged tail, and the reversed
    aggregate order, all against the oracle."""
    g = pxdata.rng(4200)
    D = 8_500
    for n in [4097, 5_500_003]:
        ranks = pxdata.zipf_ranks(g, D, n, 1.1)
        keys = (g.permutation(D)[ranks - 1] + 7).astype(kt)
        out = g.random(n) < 0.001  # outside [7, 7 + D)
        keys[out] = np.where(g.random(out.sum()) < 0.5, -5, D + 50).astype(kt)
        vals = pxdata.random_column(g, n, vt)
        cuts = np.sort(g.integers(0, n + 1, size=6))
        seg = np.concatenate([[0], cuts[:2], cuts[2:3], cuts[2:3], cuts[3:], [n]]).astype(np.int64)
        if kt == np.int64:  # a 64-bit key leaves no bits of the group code for segments
            seg = np.array([0, n], np.int64)
        for order in (0, 1):
            o_aggs = [(oracle.SUM, vals, None), (oracle.COUNT, None, None)]
            p_aggs = [(px.PX_SUM, 1, None), (px.PX_COUNT, None, None)]
            if order:
                o_aggs, p_aggs = o_aggs[::-1], p_aggs[::-1]
            want = oracle.groupby([keys], o_aggs, seg=seg)
            segmented = seg.size > 2
            res = _gb(px, [keys, vals], [0], p_aggs, (seg.size - 1) * D + 64, seg=dev(seg) if segmented else None,
                      key_range=[(7, 7 + D - 1)])
            if not segmented:
                want = oracle.groupby([keys], o_aggs)
            assert_groups_equal(res, want, 1, segmented=segmented)
