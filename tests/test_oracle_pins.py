"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each test checks the oracle against brute force on tiny inputs (a different
algorithm written in pure Python), against closed forms of the mathematics, or
against invariants that any correct result satisfies. The cases are chosen so a
plausible mistake in the oracle (a dropped term, a wrong index, an unstable
sort, a wrong sign extension, a wrong segment boundary) fails at least one.
"""
import itertools
import random

import numpy as np
import pytest

import oracle
import pxdata

M64 = 2**64 - 1
C1, C2 = 0xff51afd7ed558ccd, 0xc4ceb9fe1a85ec53  # MurmurHash3 fmix64 multipliers


def inv_fmix64(h: int) -> int:
    """Inverse of fmix64 from its structure: x ^= x >> 33 is its own inverse on 64-bit
    words (two applications cancel because 2*33 >= 64) and multiplication by an odd
    constant is undone by its inverse mod 2^64."""
    i1, i2 = pow(C1, -1, 2**64), pow(C2, -1, 2**64)
    h ^= h >> 33
    h = (h * i2) & M64
    h ^= h >> 33
    h = (h * i1) & M64
    h ^= h >> 33
    return h


def s64(u: int) -> int:
    return u - 2**64 if u >= 2**63 else u


# ---------------------------------------------------------------- hash -----

def test_fmix64_zero_fixed_point():
    # Every step of the finalizer maps 0 to 0.
    assert oracle.fmix64(0) == 0


def test_fmix64_inverse_round_trip():
    g = random.Random(1)
    xs = [g.getrandbits(64) for _ in range(2000)] + [1, 2, M64, 2**63, 2**33, 2**32 - 1]
    for x in xs:
        assert inv_fmix64(oracle.fmix64(x)) == x


def test_fmix64_avalanche():
    # A full-avalanche mixer flips ~half of the 64 output bits per flipped input bit.
    g = random.Random(2)
    flips = []
    for _ in range(300):
        x = g.getrandbits(64)
        b = g.randrange(64)
        flips.append(bin(oracle.fmix64(x) ^ oracle.fmix64(x ^ (1 << b))).count("1"))
    assert 30.0 < np.mean(flips) < 34.0


def test_part_of_range_boundaries():
    # Multiply-shift reduction: floor(x * P / 2^32) = q exactly for
    # x in [ceil(q 2^32 / P), ceil((q+1) 2^32 / P)). Build keys whose hash has a
    # chosen upper word x (via the inverse mixer) and check both ends of every bucket.
    for P in [1, 2, 3, 7, 8, 64, 1000, 1024]:
        for seed in [0, 0x9E3779B97F4A7C15]:
            for q in range(min(P, 40)):
                x_lo = -(-q * 2**32 // P)
                x_hi = -(-(q + 1) * 2**32 // P) - 1
                for x in (x_lo, x_hi):
                    h = (x << 32) | 0x1234567
                    key = s64(inv_fmix64(h) ^ seed)
                    assert oracle.part_of(key, seed, P) == q, (P, q, x)


def test_part_of_seed_is_xor_on_key():
    g = random.Random(3)
    for _ in range(200):
        k, s = s64(g.getrandbits(64)), g.getrandbits(64)
        assert oracle.part_of(k, s, 64) == oracle.part_of(s64((k & M64) ^ s), 0, 64)


def test_part_of_uniform_counts():
    # 64 buckets over 64k consecutive keys: each count within 6 sigma of 1024.
    keys = np.arange(65536, dtype=np.int64)
    p = oracle.part_of_array(keys, 0, 64)
    c = np.bincount(p, minlength=64)
    assert c.sum() == 65536 and np.all(np.abs(c - 1024) < 6 * 32)


# -------------------------------------------------------------- filter -----

@pytest.mark.parametrize("dtype", [np.int8, np.int32, np.int64])
def test_filter_brute_force(dtype):
    g = pxdata.rng(10)
    info = np.iinfo(dtype)
    for n in [0, 1, 2, 31, 33, 257]:
        col = pxdata.random_column(g, n, dtype)
        bounds = [(info.min, info.max), (-5, 5), (0, 0), (info.max, info.min),
                  (-(2**63), 2**63 - 1), (int(info.min) + 1, int(info.max))]
        if n:
            bounds.append((int(col[n // 2]), int(col[n // 2]) + 1))
        for lo, hi in bounds:
            want = [i for i in range(n) if lo <= int(col[i]) < hi]
            got = oracle.filter(col, lo, hi)
            assert got.dtype == np.int32 and got.tolist() == want


def test_filter_count_and_order_invariants():
    d = pxdata.plain(50_000, 0)
    sel = oracle.filter(d["date"], pxdata.CFG1_DATE_LO, pxdata.CFG1_DATE_HI)
    assert np.all(np.diff(sel) > 0)
    assert sel.size == int(np.count_nonzero(d["date"] < pxdata.CFG1_DATE_HI))
    # 98.005 % pass rate, within 6 sigma for 50k rows.
    p = 2506 / 2557
    assert abs(sel.size - p * 50_000) < 6 * np.sqrt(50_000 * p * (1 - p))


# ----------------------------------------------------------- partition -----

def brute_partition(cols, key_col, P, seed, sel):
    """Bucket enumeration: for q = 0..P-1 scan the input in order and take the rows
    whose key hashes to q (a different algorithm from the oracle's stable sort)."""
    rows = list(sel) if sel is not None else list(range(cols[0].size))
    part = {r: oracle.part_of(int(cols[key_col][r]), seed, P) for r in rows}
    out_rows, offsets = [], [0]
    for q in range(P):
        out_rows += [r for r in rows if part[r] == q]
        offsets.append(len(out_rows))
    return [c[np.array(out_rows, dtype=np.int64)] for c in cols], offsets


@pytest.mark.parametrize("P", [1, 2, 3, 8, 64, 1000])
def test_partition_brute_force(P):
    g = pxdata.rng(20 + P)
    for n in [0, 1, 5, 64, 300]:
        key = pxdata.random_column(g, n, np.int64, -50, 50)   # many duplicate keys
        v32 = pxdata.random_column(g, n, np.int32)
        v8 = pxdata.random_column(g, n, np.int8)
        rid = np.arange(n, dtype=np.int64)
        cols = [v32, key, v8, rid]
        for sel in [None, np.sort(g.choice(n, size=n // 2, replace=False)).astype(np.int32)
                    if n else np.zeros(0, np.int32)]:
            for seed in [0, 12345]:
                got, off = oracle.partition(cols, 1, P, seed, sel=sel)
                want, woff = brute_partition(cols, 1, P, seed, sel)
                assert off.tolist() == woff
                for a, b in zip(got, want):
                    assert a.dtype == b.dtype and np.array_equal(a, b)


def test_partition_invariants_plain_workload():
    d = pxdata.plain(30_000, 0)
    sel = oracle.filter(d["date"], pxdata.CFG1_DATE_LO, pxdata.CFG1_DATE_HI)
    rid = np.arange(30_000, dtype=np.int64)
    (key, r), off = oracle.partition([d["key"], rid], 0, 8, 0, sel=sel)
    assert off[0] == 0 and off[-1] == sel.size and np.all(np.diff(off) >= 0)
    assert sorted(r.tolist()) == sel.tolist()             # same multiset of rows
    p = oracle.part_of_array(key, 0, 8)
    for q in range(8):
        seg = slice(off[q], off[q + 1])
        assert np.all(p[seg] == q)                           # every row where its hash says
        assert np.all(np.diff(r[seg]) > 0)                   # stable
    assert np.array_equal(key, d["key"][r])


def test_partition_single_part_is_identity():
    d = pxdata.plain(5_000, 0)
    cols = [d[k] for k in ["key", "price", "date", "flag"]]
    out, off = oracle.partition(cols, 0, 1, 77)
    assert off.tolist() == [0, 5_000]
    for a, b in zip(out, cols):
        assert np.array_equal(a, b)


# ---------------------------------------------------------------- join -----

def brute_join(pk, fk, sel=None):
    rows = list(sel) if sel is not None else list(range(fk.size))
    pr, br = [], []
    for r in rows:
        for b in range(pk.size):
            if int(pk[b]) == int(fk[r]):
                pr.append(r)
                br.append(b)
    return pr, br


def test_join_brute_force_unique_and_duplicates():
    g = pxdata.rng(30)
    for nb, nprobe, dom in [(0, 10, 5), (10, 0, 5), (1, 1, 1), (20, 50, 30), (40, 100, 15),
                            (64, 200, 200)]:
        for unique in [True, False]:
            if unique:
                pk = g.permutation(max(dom, nb))[:nb].astype(np.int64) - dom // 2
            else:
                pk = pxdata.random_column(g, nb, np.int64, -(dom // 2), dom // 2)
            fk = pxdata.random_column(g, nprobe, np.int64, -(dom // 2), dom // 2)
            for sel in [None, np.sort(g.choice(nprobe, nprobe // 3, replace=False)).astype(np.int32)
                        if nprobe else np.zeros(0, np.int32)]:
                pr, br, _ = oracle.join(pk, fk, sel=sel)
                wpr, wbr = brute_join(pk, fk, sel)
                assert pr.tolist() == wpr and br.tolist() == wbr


def test_join_extreme_keys():
    pk = np.array([-(2**63), 2**63 - 1, 0, -1], dtype=np.int64)
    fk = np.array([2**63 - 1, -(2**63), 5, -1, -1], dtype=np.int64)
    pr, br, _ = oracle.join(pk, fk)
    assert pr.tolist() == [0, 1, 3, 4] and br.tolist() == [1, 0, 3, 3]


def test_join_segmented_is_per_segment_nested_loop():
    g = pxdata.rng(31)
    pk = pxdata.random_column(g, 60, np.int64, 0, 20)
    fk = pxdata.random_column(g, 150, np.int64, 0, 20)
    bseg = np.array([0, 10, 10, 45, 60], dtype=np.int64)
    pseg = np.array([0, 30, 70, 70, 150], dtype=np.int64)
    pr, br, oseg = oracle.join(pk, fk, build_seg=bseg, probe_seg=pseg)
    wpr, wbr, wseg = [], [], [0]
    for q in range(4):
        a, b = brute_join(pk[bseg[q]:bseg[q + 1]], fk[pseg[q]:pseg[q + 1]])
        wpr += [x + int(pseg[q]) for x in a]
        wbr += [x + int(bseg[q]) for x in b]
        wseg.append(len(wpr))
    assert pr.tolist() == wpr and br.tolist() == wbr and oseg.tolist() == wseg


def test_join_plain_join_closed_form():
    # pk is a permutation of 1..ndim and every fk names a pk, so every selected
    # probe row matches exactly once, at the position of its key in pk.
    d = pxdata.plain_join(2_000, 20_000)
    sel = oracle.filter(d["date"], pxdata.CFG2_DATE_LO, pxdata.CFG2_DATE_HI)
    pr, br, _ = oracle.join(d["pk"], d["fk"], sel=sel)
    pos = np.empty(2_001, dtype=np.int64)
    pos[d["pk"]] = np.arange(2_000)
    assert np.array_equal(pr, sel)
    assert np.array_equal(br, pos[d["fk"][sel]])


# ------------------------------------------------------------ group-by -----

def brute_groupby(keys, aggs, rows, seg_of=None):
    """Enumerate the distinct key tuples, then sum each aggregate over the rows of
    each tuple in Python integers reduced mod 2^64 (a different algorithm from the
    oracle's single pass over an ordered map)."""
    def key_of(r):
        return ((seg_of(r) if seg_of else 0),) + tuple(int(k[r]) for k in keys)
    distinct = sorted({key_of(r) for r in rows})
    out = []
    for t in distinct:
        members = [r for r in rows if key_of(r) == t]
        vals = []
        for op, a, b in aggs:
            if op == oracle.COUNT:
                v = len(members)
            elif op == oracle.SUM:
                v = sum(int(a[r]) for r in members)
            else:
                v = sum(int(a[r]) * int(b[r]) for r in members)
            vals.append(s64(v % 2**64))
        out.append((t, vals))
    return out


def _check_groupby(got, want, nkeys, segmented):
    assert got["ngroups"] == len(want)
    for g, (t, vals) in enumerate(want):
        if segmented:
            assert got["seg"][g] == t[0]
        for k in range(nkeys):
            assert got["keys"][k][g] == t[1 + k]
        for a, v in enumerate(vals):
            assert got["aggs"][a][g] == v


@pytest.mark.parametrize("kt", [(np.int8,), (np.int32,), (np.int64,), (np.int8, np.int8),
                                (np.int32, np.int8), (np.int64, np.int32)])
def test_groupby_brute_force(kt):
    g = pxdata.rng(40)
    for n in [0, 1, 7, 100, 400]:
        keys = [pxdata.random_column(g, n, t, -3, 3) for t in kt]
        a64 = pxdata.random_column(g, n, np.int64)          # full range: sums wrap
        a32 = pxdata.random_column(g, n, np.int32)
        b8 = pxdata.random_column(g, n, np.int8)
        aggs = [(oracle.SUM, a64, None), (oracle.COUNT, None, None),
                (oracle.SUM_MUL, a32, b8), (oracle.SUM_MUL, a64, a64), (oracle.SUM, b8, None)]
        for sel in [None, np.sort(g.choice(n, n // 2, replace=False)).astype(np.int32)
                    if n else np.zeros(0, np.int32)]:
            rows = list(sel) if sel is not None else list(range(n))
            got = oracle.groupby(keys, aggs, sel=sel)
            _check_groupby(got, brute_groupby(keys, aggs, rows), len(kt), False)


def test_groupby_segmented_brute_force():
    g = pxdata.rng(41)
    n = 200
    key = pxdata.random_column(g, n, np.int32, 0, 6)
    a = pxdata.random_column(g, n, np.int64, -1000, 1000)
    seg = np.array([0, 0, 50, 51, 130, 200], dtype=np.int64)
    got = oracle.groupby([key], [(oracle.SUM, a, None), (oracle.COUNT, None, None)], seg=seg)

    def seg_of(r):
        return int(np.searchsorted(seg, r, side="right") - 1)
    _check_groupby(got, brute_groupby([key], [(oracle.SUM, a, None), (oracle.COUNT, None, None)],
                                      list(range(n)), seg_of), 1, True)


def test_groupby_wraps_mod_2_64():
    big = np.array([2**63 - 1, 2**63 - 1, 5], dtype=np.int64)
    k = np.zeros(3, dtype=np.int32)
    got = oracle.groupby([k], [(oracle.SUM, big, None), (oracle.SUM_MUL, big, big)])
    assert got["aggs"][0][0] == s64((2 * (2**63 - 1) + 5) % 2**64)
    assert got["aggs"][1][0] == s64((2 * (2**63 - 1) ** 2 + 25) % 2**64)


def test_groupby_max_groups_truncates_but_counts():
    k = np.arange(10, dtype=np.int32)
    got = oracle.groupby([k], [(oracle.COUNT, None, None)], max_groups=4)
    assert got["ngroups"] == 10 and got["keys"][0].tolist() == [0, 1, 2, 3]


def test_groupby_invariants_and_constant_key():
    d = pxdata.plain(40_000, 0)
    g = oracle.groupby([d["flag"], d["status"]],
                       [(oracle.SUM, d["price"], None), (oracle.COUNT, None, None)])
    assert g["ngroups"] == 8
    assert int(g["aggs"][1].sum()) == 40_000
    assert int(g["aggs"][0].sum()) == int(d["price"].sum())
    c = oracle.groupby([np.zeros(40_000, np.int8)],
                       [(oracle.SUM, d["price"], None), (oracle.SUM_MUL, d["price"], d["qty"])])
    assert c["ngroups"] == 1 and c["aggs"][0][0] == int(d["price"].sum())
    assert c["aggs"][1][0] == int((d["price"] * d["qty"]).sum())


# ----------------------------------------------------------- pipelines -----

def test_at_scale_partitioned_equals_unpartitioned():
    # The exchange must not change the answer: per-partition join + Partial
    # aggregation + Final merge equals the unpartitioned join + aggregation.
    d = pxdata.plain_at_scale(5_000, 100_000, nattr=300)
    r = oracle.pipeline_at_scale(d, 64)
    pr, br, _ = oracle.join(d["pk"], d["fk"])
    g = oracle.groupby([d["attr"][br]], [(oracle.SUM, d["amount"][pr], None),
                                         (oracle.COUNT, None, None)])
    f = r["final"]
    assert f["ngroups"] == g["ngroups"]
    assert np.array_equal(f["keys"][0], g["keys"][0])
    for a in range(2):
        assert np.array_equal(f["aggs"][a], g["aggs"][a])
    assert int(f["aggs"][1].sum()) == 100_000            # every fact row joins once
    assert int(r["partial"]["aggs"][1].sum()) == 100_000


def test_plain_pipeline_invariants():
    d = pxdata.plain(30_000, 0)
    r = oracle.pipeline_plain(d, pxdata.CFG1_DATE_LO, pxdata.CFG1_DATE_HI, 8)
    g = r["groups"]
    assert g["ngroups"] == 8
    assert int(g["aggs"][3].sum()) == r["sel"].size
    assert int(g["aggs"][0].sum()) == int(d["price"][r["sel"]].sum())
    assert int(g["aggs"][1].sum()) == int((d["price"][r["sel"]] * d["qty"][r["sel"]]).sum())


def test_zipf_head_share():
    # Closed form of the generator's skew: P(rank 1) = 1 / H_{N,s}.
    d = pxdata.plain_at_scale(200_000, 400_000, nattr=10)
    top = np.bincount(np.unique(d["fk"], return_inverse=True)[1]).max()
    H = float(np.sum(np.arange(1, 200_001, dtype=np.float64) ** -1.1))
    p = 1 / H
    assert abs(top - p * 400_000) < 6 * np.sqrt(400_000 * p * (1 - p))


# ------------------------------------------------ composed pipelines -----

def _brute_groups(rows):
    """rows: (group key, tuple of addends); per key the wrapped sums, keys ascending."""
    acc = {}
    for k, vals in rows:
        cur = acc.setdefault(k, [0] * len(vals))
        for a, x in enumerate(vals):
            cur[a] = (cur[a] + x) & M64
    keys = sorted(acc)
    return keys, [[s64(acc[k][a]) for k in keys] for a in range(len(acc[keys[0]]) if keys else 0)]


def _assert_groups(g, keys, sums):
    assert g["ngroups"] == len(keys)
    assert g["keys"][0].tolist() == keys
    for a, col in enumerate(sums):
        assert g["aggs"][a].tolist() == col


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fragment_pipeline_brute_force(seed):
    # Nested loops over (fact row, dim row) straight from the definition: keep
    # lo <= date < hi, match key = pk, group by the dim row's attr; SUM(price),
    # SUM(price * qty), COUNT(*) all from the FACT row.
    d = pxdata.fragment(300, 40, 6, seed=70 + seed)
    d["date"][:5] = [pxdata.CFG2_DATE_LO - 1, pxdata.CFG2_DATE_LO, pxdata.CFG2_DATE_HI - 1, pxdata.CFG2_DATE_HI, 0]
    rows = []
    for i in range(d["key"].size):
        if not (pxdata.CFG2_DATE_LO <= d["date"][i] < pxdata.CFG2_DATE_HI):
            continue
        for j in range(d["pk"].size):
            if d["pk"][j] == d["key"][i]:
                p, q = int(d["price"][i]), int(d["qty"][i])
                rows.append((int(d["attr"][j]), (p, p * q, 1)))
    keys, sums = _brute_groups(rows)
    r = oracle.pipeline_fragment(d, pxdata.CFG2_DATE_LO, pxdata.CFG2_DATE_HI)
    _assert_groups(r["groups"], keys, sums)
    assert 0 < len(rows) < d["key"].size  # some rows filtered or unmatched, some kept


def test_wide_join_pipeline_brute_force():
    # Build side = the dim rows with attr below the bound; SUM(amount),
    # SUM(price * qty), COUNT(*) from the fact row, grouped by the build row's attr.
    d = pxdata.wide_at_scale(200, 3000, nattr=50, build_attr_below=10, seed=9)
    rows = []
    for i in range(d["fk"].size):
        for j in range(d["pk_b"].size):
            if d["pk_b"][j] == d["fk"][i]:
                p, q = int(d["price"][i]), int(d["qty"][i])
                rows.append((int(d["attr_b"][j]), (int(d["amount"][i]), p * q, 1)))
    keys, sums = _brute_groups(rows)
    _assert_groups(oracle.pipeline_wide_join(d), keys, sums)
    assert 0 < len(rows) < d["fk"].size


def test_at_scale_final_brute_force():
    # Final groups of the exchange -> join -> Partial -> Final chain equal a nested
    # loop over the unpartitioned rows: SUM(amount) and COUNT(*) by the dim attr.
    d = pxdata.plain_at_scale(150, 2000, nattr=7, seed=11)
    rows = []
    for i in range(d["fk"].size):
        for j in range(d["pk"].size):
            if d["pk"][j] == d["fk"][i]:
                rows.append((int(d["attr"][j]), (int(d["amount"][i]), 1)))
    keys, sums = _brute_groups(rows)
    _assert_groups(oracle.pipeline_at_scale(d, 8)["final"], keys, sums)
