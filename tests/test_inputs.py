"""The seeded input recipes (pxdata): column types, ranges and the properties the
parity tests and closed forms rely on (every plain-join key names one dimension
row, about 5 % of fragment keys name none, the wide join keeps about 10 % of the
dimension), plus reproducibility from the seed. No GPU."""
import numpy as np
import pytest

import pxdata


def test_plain_columns_types_and_ranges():
    d = pxdata.plain(200_000, 0)
    want = {"key": (np.int64, 0, 2**20 - 1), "price": (np.int64, 100, 10**7), "qty": (np.int64, 1, 50),
            "date": (np.int32, 0, pxdata.DATE_DAYS - 1), "flag": (np.int8, 0, 3), "status": (np.int8, 0, 1)}
    assert list(d) == list(want)
    for k, (dt, lo, hi) in want.items():
        assert d[k].dtype == dt and d[k].flags.c_contiguous
        assert d[k].min() >= lo and d[k].max() <= hi
        assert d[k].min() <= lo + (hi - lo) // 50 and d[k].max() >= hi - (hi - lo) // 50  # spans its range
    # the filter bound keeps 2506 of 2557 days
    keep = (d["date"] < pxdata.CFG1_DATE_HI).mean()
    assert abs(keep - 2506 / 2557) < 0.002


def test_plain_join_every_key_names_exactly_one_pk():
    d = pxdata.plain_join(20_000, 300_000, 25, seed=2)
    assert np.array_equal(np.sort(d["pk"]), np.arange(1, 20_001))           # a permutation of 1..ndim
    assert d["fk"].min() >= 1 and d["fk"].max() <= 20_000
    assert d["attr"].min() >= 0 and d["attr"].max() <= 24
    window = ((d["date"] >= pxdata.CFG2_DATE_LO) & (d["date"] < pxdata.CFG2_DATE_HI)).mean()
    assert abs(window - 767 / 2557) < 0.005


def test_fragment_about_five_percent_of_keys_miss():
    d = pxdata.fragment(400_000, 20_000, 37, seed=5)
    assert np.array_equal(np.sort(d["pk"]), np.arange(1, 20_001))
    miss = (d["key"] > 20_000).mean()
    assert abs(miss - 1000 / 21_000) < 0.003                                 # keys U[1, nbuild + nbuild // 20]
    assert d["attr"].max() <= 36 and d["key"].min() >= 1


def test_fragment_sizes_follow_their_log_uniform_bounds():
    s = pxdata.fragment_sizes(512, seed=4)
    assert s["nfact"].min() >= 10_000 and s["nfact"].max() < 4_000_000
    assert s["nbuild"].min() >= 1_000 and s["nbuild"].max() < 1_000_000
    assert s["ngroups"].min() >= 4 and s["ngroups"].max() < 100_000
    # log-uniform: the median sits near the geometric mean of the bounds
    assert abs(np.log(np.median(s["nfact"])) - 0.5 * np.log(1e4 * 4e6)) < 0.35
    assert 2.0e8 < s["nfact"].sum() < 5.5e8
    small = pxdata.fragment_sizes(16, seed=4, scale=0.01)
    assert small["nfact"].max() < 40_000 and small["nbuild"].min() >= 10


def test_wide_join_keeps_about_a_tenth_of_the_dimension():
    d = pxdata.wide_at_scale(50_000, 200_000, nattr=10_000, build_attr_below=1_000, seed=6)
    assert abs(d["pk_b"].size / 50_000 - 0.1) < 0.01
    assert d["attr_b"].max() < 1_000
    assert np.isin(d["pk_b"], d["pk"]).all()
    assert d["price"].min() >= 100 and d["qty"].max() <= 50


@pytest.mark.parametrize("make", [lambda s: pxdata.plain(5_000, s), lambda s: pxdata.plain_join(500, 5_000, seed=s),
                                  lambda s: pxdata.plain_at_scale(500, 5_000, nattr=10, seed=s),
                                  lambda s: pxdata.fragment(5_000, 500, 7, seed=s)])
def test_same_seed_same_arrays_other_seed_other_arrays(make):
    a, b, c = make(11), make(11), make(12)
    assert all(np.array_equal(a[k], b[k]) for k in a)
    assert any(not np.array_equal(a[k], c[k]) for k in a)
