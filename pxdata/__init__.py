"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only draws random columns. It holds none of the method's arithmetic
(no hashing, no partitioning, no joins, no aggregation), so both the CPU oracle
and the CUDA path can consume the same arrays without sharing any code.

The shapes follow the TPC-H-like operator workloads of the paper (Sec. 2.3 and
Sec. 3.4: a scan-filter-aggregate query like Q1, a fact/dimension hash join
followed by an aggregation like Q5/Q9) but are purely synthetic: no TPC-H data,
dbgen output or query text is used. All draws use numpy's PCG64 generator, one
draw per column in the order listed in each function.

Every array is a fresh, C-contiguous numpy array. Column dtypes are the Arrow
fixed-width types the operators take: int8, int32 and int64 (decimals are
int64 fixed-point, scale 2 for prices and amounts).
"""
from __future__ import annotations

import numpy as np

DATE_DAYS = 2557  # 7 years of day offsets 0..2556

# Filter bounds (half-open [lo, hi)) of the workloads.
CFG1_DATE_LO = -(2**31)      # date < 2506 keeps 2506/2557 = 98.005 % of rows
CFG1_DATE_HI = 2506
CFG2_DATE_LO = 895           # a 767-day window keeps 767/2557 = 29.996 %
CFG2_DATE_HI = 1662

CFG1_PARTS = 8
CFG3_PARTS = 64


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def plain(n: int = 1_000_000, seed: int = 0) -> dict:
    """Scan-filter-partition-aggregate batch (the 1M-row 'plain' workload).

    key int64 U[0, 2^20); price int64 U[100, 10^7] (scale 2); qty int64 U[1, 50];
    date int32 U[0, 2557); flag int8 U{0..3}; status int8 U{0, 1}.
    """
    g = _rng(seed)
    return {
        "key": g.integers(0, 2**20, size=n, dtype=np.int64),
        "price": g.integers(100, 10**7, size=n, dtype=np.int64, endpoint=True),
        "qty": g.integers(1, 50, size=n, dtype=np.int64, endpoint=True),
        "date": g.integers(0, DATE_DAYS, size=n, dtype=np.int32),
        "flag": g.integers(0, 4, size=n, dtype=np.int8),
        "status": g.integers(0, 2, size=n, dtype=np.int8),
    }


def plain_join(ndim: int = 200_000, nfact: int = 6_000_000, nattr: int = 25,
               seed: int = 2) -> dict:
    """Dimension/fact pair of the plain-join workload.

    dim: pk int64 = seeded permutation of 1..ndim, attr int32 U[0, nattr).
    fact: fk int64 U[1, ndim] (every fk names a pk), amount int64 U[100, 10^6]
    (scale 2), date int32 U[0, 2557).
    """
    g = _rng(seed)
    pk = g.permutation(ndim).astype(np.int64) + 1
    attr = g.integers(0, nattr, size=ndim, dtype=np.int32)
    fk = g.integers(1, ndim, size=nfact, dtype=np.int64, endpoint=True)
    amount = g.integers(100, 10**6, size=nfact, dtype=np.int64, endpoint=True)
    date = g.integers(0, DATE_DAYS, size=nfact, dtype=np.int32)
    return {"pk": pk, "attr": attr, "fk": fk, "amount": amount, "date": date}


def zipf_ranks(g: np.random.Generator, nranks: int, size: int, s: float) -> np.ndarray:
    """Draw ranks 1..nranks with P(r) proportional to r^-s by inverse CDF."""
    w = np.arange(1, nranks + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = g.random(size)
    r = np.searchsorted(cdf, u, side="right")
    np.minimum(r, nranks - 1, out=r)
    return r.astype(np.int64) + 1


def plain_at_scale(ndim: int = 2_000_000, nfact: int = 60_000_000, nattr: int = 10_000,
                   zipf_s: float = 1.1, seed: int = 3) -> dict:
    """Skewed dimension/fact pair of the at-scale workload.

    dim: pk int64 = seeded permutation of 1..ndim, attr int32 U[0, nattr).
    fact: fk int64 = pk_of_rank[r] with r ~ Zipf(s) over ranks 1..ndim (the
    rank-to-pk map is a second seeded permutation), amount int64 U[100, 10^6]
    (scale 2), date int32 U[0, 2557) (not filtered in this workload).
    With s = 1.1 and ndim = 2M the hottest key holds about 12.1 % of fact rows.
    """
    g = _rng(seed)
    pk = g.permutation(ndim).astype(np.int64) + 1
    attr = g.integers(0, nattr, size=ndim, dtype=np.int32)
    pk_of_rank = g.permutation(ndim).astype(np.int64) + 1
    r = zipf_ranks(g, ndim, nfact, zipf_s)
    fk = pk_of_rank[r - 1]
    amount = g.integers(100, 10**6, size=nfact, dtype=np.int64, endpoint=True)
    date = g.integers(0, DATE_DAYS, size=nfact, dtype=np.int32)
    return {"pk": pk, "attr": attr, "fk": fk, "amount": amount, "date": date}


def wide_at_scale(ndim: int = 2_000_000, nfact: int = 60_000_000, nattr: int = 10_000, build_attr_below: int = 1_000,
                  seed: int = 6) -> dict:
    """Selective join over a wide fact (the late-materialization workload).

    The at-scale pair (same recipe, this seed) plus fact price int64 U[100, 10^7]
    (scale 2) and qty int64 U[1, 50], drawn after it. The build side is the
    dimension rows with attr < build_attr_below (about 10 % of them), so only the
    fact rows whose key names one of those survive the join.
    """
    d = plain_at_scale(ndim, nfact, nattr, seed=seed)
    g = _rng(seed + 1000)
    d["price"] = g.integers(100, 10**7, size=nfact, dtype=np.int64, endpoint=True)
    d["qty"] = g.integers(1, 50, size=nfact, dtype=np.int64, endpoint=True)
    keep = d["attr"] < build_attr_below
    d["pk_b"] = d["pk"][keep]
    d["attr_b"] = d["attr"][keep]
    return d


def _log_uniform_int(g: np.random.Generator, lo: int, hi: int, size: int) -> np.ndarray:
    return np.floor(np.exp(g.uniform(np.log(lo), np.log(hi), size=size))).astype(np.int64)


def fragment_sizes(nfrags: int = 512, seed: int = 4, scale: float = 1.0) -> dict:
    """Sizes of the batched-fragments workload: per fragment, fact rows log-uniform
    in [10^4, 4*10^6], build rows log-uniform in [10^3, 10^6] and group-key domain
    log-uniform in [4, 10^5], each bound multiplied by `scale` (at least 1; tests
    use small scales). Drawn in that order."""
    g = _rng(seed)
    lo = lambda x: max(1, int(x * scale))
    return {"nfact": _log_uniform_int(g, lo(1e4), lo(4e6), nfrags),
            "nbuild": _log_uniform_int(g, lo(1e3), lo(1e6), nfrags),
            "ngroups": _log_uniform_int(g, 4, max(5, lo(1e5)), nfrags)}


def fragment(nfact: int, nbuild: int, ngroups: int, seed: int) -> dict:
    """One fragment of the batched workload: a dimension and a fact batch with the
    plain workload's column types.

    dim: pk int64 = seeded permutation of 1..nbuild, attr int32 U[0, ngroups).
    fact: key int64 U[1, nbuild + nbuild // 20] (about 5 % of keys name no pk),
    price int64 U[100, 10^7] (scale 2), qty int64 U[1, 50], date int32 U[0, 2557).
    """
    g = _rng(seed)
    pk = g.permutation(nbuild).astype(np.int64) + 1
    attr = g.integers(0, ngroups, size=nbuild, dtype=np.int32)
    key = g.integers(1, nbuild + nbuild // 20, size=nfact, dtype=np.int64, endpoint=True)
    price = g.integers(100, 10**7, size=nfact, dtype=np.int64, endpoint=True)
    qty = g.integers(1, 50, size=nfact, dtype=np.int64, endpoint=True)
    date = g.integers(0, DATE_DAYS, size=nfact, dtype=np.int32)
    return {"pk": pk, "attr": attr, "key": key, "price": price, "qty": qty, "date": date}


def random_column(g: np.random.Generator, n: int, dtype, lo=None, hi=None) -> np.ndarray:
    """A column of n values of `dtype` uniform in [lo, hi] (default: the full type range)."""
    info = np.iinfo(dtype)
    lo = info.min if lo is None else lo
    hi = info.max if hi is None else hi
    return g.integers(lo, hi, size=n, dtype=dtype, endpoint=True)


def rng(seed: int) -> np.random.Generator:
    """The generator every test draws its small random cases from."""
    return _rng(seed)
