"""CPU oracle for the px operators: TEST INFRASTRUCTURE ONLY.

Plain, slow, single-threaded statements of what the GPU path computes (filter,
hash partition, equi-join, hash aggregation and the three workload pipelines),
compiled from ``px_oracle.cpp`` with g++ and called through ctypes on numpy
arrays. Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline / reference arm may import this package; the product library never
does. It imports nothing from the CUDA package.

Each function names the operator statement of the paper it follows (section
numbers of "Accelerating Presto with GPUs"); the readings taken where the paper
is silent (hash function, stable order, half-open predicate, output order) are
stated in ``px_oracle.cpp``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "px_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
# A prebuilt oracle library to load instead (the mutation tests point this at
# deliberately broken copies to show the pins reject them).
_LIB_OVERRIDE = os.environ.get("PX_ORACLE_LIB")

COUNT, SUM, SUM_MUL = 0, 1, 2

_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ -O2 (single-threaded, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        if _LIB_OVERRIDE:
            lib = ctypes.CDLL(_LIB_OVERRIDE)
        else:
            build()
            lib = ctypes.CDLL(_LIB)
        P, I32, I64, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        lib.orc_fmix64.argtypes = [U64]
        lib.orc_fmix64.restype = U64
        lib.orc_part_of.argtypes = [I64, U64, I32]
        lib.orc_part_of.restype = I32
        lib.orc_filter.argtypes = [P, I32, I64, I64, I64, P]
        lib.orc_filter.restype = I64
        lib.orc_partition.argtypes = [I32, P, P, I64, I32, P, I64, I32, U64, P, P]
        lib.orc_partition.restype = I32
        lib.orc_join.argtypes = [P, I64, P, P, I64, P, I64, P, I32, I64, P, P, P]
        lib.orc_join.restype = I64
        lib.orc_groupby.argtypes = [I64, P, I64, P, I32, I32, P, P, I32, P, P, P, P, P,
                                    I64, P, P, P]
        lib.orc_groupby.restype = I64
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _ptrs(arrays):
    arr = (ctypes.c_void_p * max(1, len(arrays)))()
    for i, a in enumerate(arrays):
        arr[i] = a.ctypes.data
    return arr


def _widths(arrays):
    return np.array([a.dtype.itemsize for a in arrays], dtype=np.int32)


def _c(a, dtype=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a)
    if dtype is not None and a.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {a.dtype}")
    return a


def fmix64(x: int) -> int:
    """MurmurHash3 fmix64 of a 64-bit word (partition hash reading)."""
    return int(_load().orc_fmix64(int(x) & (2**64 - 1)))


def part_of(key: int, seed: int, nparts: int) -> int:
    """Destination partition of one key (exchange producer, Sec. 3.3.2)."""
    return int(_load().orc_part_of(int(key), int(seed) & (2**64 - 1), int(nparts)))


def part_of_array(keys: np.ndarray, seed: int, nparts: int) -> np.ndarray:
    lib = _load()
    return np.array([lib.orc_part_of(int(k), seed, nparts) for k in keys], dtype=np.int32)


def filter(col: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """FilterProject's predicate lo <= col < hi (Sec. 3.2): ascending int32 row list."""
    col = _c(col)
    sel = np.empty(max(1, col.size), dtype=np.int32)
    n = _load().orc_filter(_ptr(col), col.dtype.itemsize, col.size, int(lo), int(hi), _ptr(sel))
    return sel[:n].copy()


def partition(cols: list, key_col: int, nparts: int, seed: int = 0, sel=None):
    """Hash repartition into nparts segments (PartitionedOutput, Sec. 3.1/3.3.2).

    Returns (list of output columns, offsets int64[nparts+1])."""
    cols = [_c(c) for c in cols]
    sel = _c(sel, np.int32)
    m = sel.size if sel is not None else cols[0].size
    outs = [np.empty(max(1, m), dtype=c.dtype) for c in cols]
    offsets = np.empty(nparts + 1, dtype=np.int64)
    _load().orc_partition(len(cols), _ptr(_widths(cols)), _ptrs(cols), cols[0].size, key_col,
                          _ptr(sel), m if sel is not None else 0, nparts,
                          int(seed) & (2**64 - 1), _ptrs(outs), _ptr(offsets))
    return [o[:m].copy() for o in outs], offsets


def join(pk: np.ndarray, fk: np.ndarray, sel=None, build_seg=None, probe_seg=None):
    """Inner equi-join fk = pk (join pipelines of Sec. 3, per partition when segmented).

    Returns (probe_rows int32, build_rows int32, out_seg int64[nsegs+1] or None)."""
    pk = _c(pk, np.int64)
    fk = _c(fk, np.int64)
    sel = _c(sel, np.int32)
    nsegs = 0
    if build_seg is not None:
        build_seg = _c(build_seg, np.int64)
        probe_seg = _c(probe_seg, np.int64)
        nsegs = build_seg.size - 1
    lib = _load()
    m = sel.size if sel is not None else fk.size
    out_seg = np.zeros(max(nsegs, 1) + 1, dtype=np.int64)
    args = (_ptr(pk), pk.size, _ptr(build_seg), _ptr(fk), fk.size, _ptr(sel),
            m if sel is not None else 0, _ptr(probe_seg), nsegs)
    dummy = np.empty(1, dtype=np.int32)
    total = lib.orc_join(*args, 0, _ptr(dummy), _ptr(dummy), None)
    pr = np.empty(max(1, total), dtype=np.int32)
    br = np.empty(max(1, total), dtype=np.int32)
    lib.orc_join(*args, total, _ptr(pr), _ptr(br), _ptr(out_seg))
    return pr[:total].copy(), br[:total].copy(), (out_seg if nsegs > 0 else None)


def groupby(keys: list, aggs: list, sel=None, seg=None, max_groups=None):
    """Hash aggregation (HashAggregation, Sec. 3.2).

    keys: list of key columns. aggs: list of (op, a, b) with op in COUNT/SUM/SUM_MUL
    and a, b numpy columns (None where unused). seg: optional segment offsets over
    positions (Partial mode per partition). Returns dict with 'seg' (int32, or None),
    'keys' (list of int64 arrays), 'aggs' (list of int64 arrays), groups in ascending
    (segment, key...) order."""
    keys = [_c(k) for k in keys]
    sel = _c(sel, np.int32)
    nrows = keys[0].size if keys else (aggs[0][1].size if aggs and aggs[0][1] is not None else 0)
    seg = _c(seg, np.int64)
    nsegs = 0 if seg is None else seg.size - 1
    ops = np.array([a[0] for a in aggs], dtype=np.int32)
    filler = np.zeros(1, dtype=np.int64)
    acols = [_c(a[1]) if a[1] is not None else filler for a in aggs]
    bcols = [_c(a[2]) if a[2] is not None else filler for a in aggs]
    lib = _load()
    m = sel.size if sel is not None else nrows
    args = (nrows, _ptr(sel), m if sel is not None else 0, _ptr(seg), nsegs,
            len(keys), _ptr(_widths(keys)), _ptrs(keys), len(aggs), _ptr(ops),
            _ptr(_widths(acols)), _ptrs(acols), _ptr(_widths(bcols)), _ptrs(bcols))
    if max_groups is None:
        d = np.empty(1, dtype=np.int64)
        max_groups = lib.orc_groupby(*args, 0, None, _ptr(d), _ptr(d))
    G = max(1, int(max_groups))
    out_seg = np.empty(G, dtype=np.int32)
    out_keys = np.empty(max(1, len(keys)) * G, dtype=np.int64)
    out_aggs = np.empty(max(1, len(aggs)) * G, dtype=np.int64)
    ng = lib.orc_groupby(*args, G, _ptr(out_seg), _ptr(out_keys), _ptr(out_aggs))
    w = min(ng, int(max_groups))
    return {
        "ngroups": int(ng),
        "seg": out_seg[:w].copy() if nsegs > 0 else None,
        "keys": [out_keys[k * G:k * G + w].copy() for k in range(len(keys))],
        "aggs": [out_aggs[a * G:a * G + w].copy() for a in range(len(aggs))],
    }


# ---------------------------------------------------------------------------
# The three workload pipelines, operator by operator.
# ---------------------------------------------------------------------------

def pipeline_plain(d: dict, lo: int, hi: int, nparts: int, seed: int = 0) -> dict:
    """Scan-filter-exchange-aggregate (Q1-like, Sec. 2.3): filter date in [lo, hi),
    hash-partition on key, group by (flag, status) with SUM(price), SUM(price*qty),
    SUM(qty), COUNT(*)."""
    sel = filter(d["date"], lo, hi)
    names = ["key", "price", "qty", "date", "flag", "status"]
    parts, offsets = partition([d[n] for n in names], 0, nparts, seed, sel=sel)
    p = dict(zip(names, parts))
    g = groupby([p["flag"], p["status"]],
                [(SUM, p["price"], None), (SUM_MUL, p["price"], p["qty"]),
                 (SUM, p["qty"], None), (COUNT, None, None)])
    return {"sel": sel, "parts": p, "offsets": offsets, "groups": g}


def pipeline_join(d: dict, lo: int, hi: int) -> dict:
    """Filter-join-aggregate (Q5/Q9-like, Sec. 3.4): filter fact.date in [lo, hi),
    join fk = pk, group by dim.attr with SUM(amount), COUNT(*)."""
    sel = filter(d["date"], lo, hi)
    pr, br, _ = join(d["pk"], d["fk"], sel=sel)
    amount = d["amount"][pr]
    attr = d["attr"][br]
    g = groupby([attr], [(SUM, amount, None), (COUNT, None, None)])
    return {"sel": sel, "probe_rows": pr, "build_rows": br, "groups": g}


def pipeline_fragment(d: dict, lo: int, hi: int) -> dict:
    """One batched fragment (FilterProject -> join probe -> Single-mode
    HashAggregation, Sec. 3.2 operators in a Q5/Q9-like plan, Sec. 3.4): keep fact
    rows with lo <= date < hi, join key = pk, group by dim.attr with SUM(price),
    SUM(price * qty), COUNT(*). Groups in ascending attr order."""
    sel = filter(d["date"], lo, hi)
    pr, br, _ = join(d["pk"], d["key"], sel=sel)
    attr = d["attr"][br]
    g = groupby([attr], [(SUM, d["price"][pr], None), (SUM_MUL, d["price"][pr], d["qty"][pr]),
                         (COUNT, None, None)])
    return {"sel": sel, "probe_rows": pr, "build_rows": br, "groups": g}


def pipeline_wide_join(d: dict) -> dict:
    """Selective join over a wide fact, aggregated (the answer of both the eager and
    the late-materialization plans, Sec. 2.3): join fk = pk over the build rows
    (pk_b, attr_b), group by attr with SUM(amount), SUM(price * qty), COUNT(*).
    Single mode over unpartitioned rows; groups in ascending attr order."""
    pr, br, _ = join(d["pk_b"], d["fk"])
    attr = d["attr_b"][br]
    return groupby([attr], [(SUM, d["amount"][pr], None), (SUM_MUL, d["price"][pr], d["qty"][pr]),
                            (COUNT, None, None)])


def pipeline_at_scale(d: dict, nparts: int, seed: int = 0) -> dict:
    """Exchange-join-aggregate at scale (Sec. 3.3 exchange feeding per-partition joins
    and Partial aggregation, then a Final merge, Sec. 3.2): partition dim on pk and
    fact on fk into nparts, join per partition, group by attr per partition
    (Partial), merge the partials by attr (Final)."""
    dparts, doff = partition([d["pk"], d["attr"]], 0, nparts, seed)
    fparts, foff = partition([d["fk"], d["amount"], d["date"]], 0, nparts, seed)
    pr, br, jseg = join(dparts[0], fparts[0], build_seg=doff, probe_seg=foff)
    amount = fparts[1][pr]
    attr = dparts[1][br]
    partial = groupby([attr], [(SUM, amount, None), (COUNT, None, None)], seg=jseg)
    final = groupby([partial["keys"][0]],
                    [(SUM, partial["aggs"][0], None), (SUM, partial["aggs"][1], None)])
    return {"dim_offsets": doff, "fact_offsets": foff, "join_offsets": jseg,
            "dim_parts": dparts, "fact_parts": fparts, "probe_rows": pr, "build_rows": br,
            "partial": partial, "final": final}
