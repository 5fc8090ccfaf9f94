"""The C ABI without a GPU: libpx.so builds, loads, exports every function that
include/px.h declares, and rejects bad arguments on the host (before any CUDA
call) with the documented status codes and a message."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:px_status|size_t|uint64_t|const char\*)\s+(px_\w+)\s*\(", text, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2606_24647_gb300 import build
    path = build.build()
    import paper_2606_24647_gb300 as pxm
    return pxm.load(path)


def test_header_declares_the_five_operators():
    names = set(declared_functions())
    for op in ["px_filter", "px_partition", "px_join_build", "px_join_probe", "px_groupby_agg"]:
        assert op in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2606_24647_gb300 import LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (px_\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_binding_declares_every_symbol():
    import paper_2606_24647_gb300 as pxm
    assert sorted(pxm.EXPORTED) == sorted(declared_functions())


FAKE = 0x7f0000000000  # 16-byte aligned, never dereferenced: every case fails a host check first


def _batch(pxm, types, nrows, ptrs=None):
    cols = (pxm.px_col * len(types))(*[pxm.px_col(t, 0, (ptrs or [FAKE + 4096 * i for i in range(len(types))])[i])
                                       for i, t in enumerate(types)])
    b = pxm.px_batch(len(types), 0, ctypes.cast(cols, ctypes.POINTER(pxm.px_col)), nrows, None)
    b._keep = cols
    return b


def test_workspace_sizes_are_monotone(lib):
    for f, args in [(lib.px_filter_ws_bytes, [(10,), (10_000,), (10_000_000,)]),
                    (lib.px_partition_ws_bytes, [(10, 8), (10_000, 8), (10_000, 64), (10_000_000, 64)]),
                    (lib.px_join_probe_ws_bytes, [(10,), (10_000,), (10_000_000,)]),
                    (lib.px_groupby_ws_bytes, [(10, 1), (10, 1000), (10, 100_000)])]:
        sizes = [f(*a) for a in args]
        assert sizes == sorted(sizes) and sizes[0] >= 256
    assert lib.px_join_table_bytes(1000, 0) < lib.px_join_table_bytes(2000, 0)
    assert lib.px_join_table_bytes(1000, 64) >= 16 * 2 * 1000


def test_host_checks(lib):
    import paper_2606_24647_gb300 as pxm
    ws = FAKE
    wsz = 1 << 30
    # filter: null column, unknown type, misaligned data, null outputs
    assert lib.px_filter(None, 10, None, 0, 1, FAKE, FAKE, ws, wsz, None) == pxm.PX_ERR_INVALID
    bad = pxm.px_col(3, 0, FAKE)
    assert lib.px_filter(ctypes.byref(bad), 10, None, 0, 1, FAKE, FAKE, ws, wsz, None) == pxm.PX_ERR_INVALID
    assert "type" in pxm.last_error()
    mis = pxm.px_col(pxm.PX_I32, 0, FAKE + 4)
    assert lib.px_filter(ctypes.byref(mis), 10, None, 0, 1, FAKE, FAKE, ws, wsz, None) == pxm.PX_ERR_INVALID
    assert "aligned" in pxm.last_error()
    ok = pxm.px_col(pxm.PX_I32, 0, FAKE)
    assert lib.px_filter(ctypes.byref(ok), 10, None, 0, 1, None, FAKE, ws, wsz, None) == pxm.PX_ERR_INVALID
    assert lib.px_filter(ctypes.byref(ok), 10, None, 0, 1, FAKE, FAKE, ws, 16, None) == pxm.PX_ERR_INVALID
    assert "workspace" in pxm.last_error()
    # partition: non-int64 key, bad nparts, column count / type mismatch
    inb = _batch(pxm, [pxm.PX_I64, pxm.PX_I32], 100)
    outb = _batch(pxm, [pxm.PX_I64, pxm.PX_I32], 100)
    r = lib.px_partition(ctypes.byref(inb), 1, None, None, 8, 0, ctypes.byref(outb), FAKE, ws, wsz, None)
    assert r == pxm.PX_ERR_INVALID
    for P in [0, pxm_max_parts() + 1]:
        r = lib.px_partition(ctypes.byref(inb), 0, None, None, P, 0, ctypes.byref(outb), FAKE, ws, wsz, None)
        assert r == pxm.PX_ERR_UNSUPPORTED
    out_bad = _batch(pxm, [pxm.PX_I64, pxm.PX_I64], 100)
    r = lib.px_partition(ctypes.byref(inb), 0, None, None, 8, 0, ctypes.byref(out_bad), FAKE, ws, wsz, None)
    assert r == pxm.PX_ERR_INVALID
    small = _batch(pxm, [pxm.PX_I64, pxm.PX_I32], 50)
    r = lib.px_partition(ctypes.byref(inb), 0, None, None, 8, 0, ctypes.byref(small), FAKE, ws, wsz, None)
    assert r == pxm.PX_ERR_INVALID and "capacity" in pxm.last_error()
    # selection pointer without its count
    r = lib.px_partition(ctypes.byref(inb), 0, FAKE, None, 8, 0, ctypes.byref(outb), FAKE, ws, wsz, None)
    assert r == pxm.PX_ERR_INVALID
    # join build: table too small, segments without offsets
    b = _batch(pxm, [pxm.PX_I64], 100)
    assert lib.px_join_build(ctypes.byref(b), 0, None, 0, 1, -1, FAKE, 64, ws, wsz, None) == pxm.PX_ERR_INVALID
    assert lib.px_join_build(ctypes.byref(b), 0, None, 4, 1, -1, FAKE, 1 << 30, ws, wsz, None) == pxm.PX_ERR_INVALID
    # group-by: too many key bits with segments, wrong output arity
    g_in = _batch(pxm, [pxm.PX_I64, pxm.PX_I64], 100)
    g_out = _batch(pxm, [pxm.PX_I64, pxm.PX_I64], 100)
    keys = (ctypes.c_int32 * 1)(0)
    aggs = (pxm.px_agg * 1)(pxm.px_agg(pxm.PX_SUM, 1, -1))
    r = lib.px_groupby_agg(ctypes.byref(g_in), keys, 1, aggs, 1, None, None, FAKE, 4, None, 100,
                           ctypes.byref(g_out), None, FAKE, ws, wsz, None)
    assert r == pxm.PX_ERR_UNSUPPORTED and "bits" in pxm.last_error()
    r = lib.px_groupby_agg(ctypes.byref(g_in), keys, 1, aggs, 1, None, None, None, 0, None, 100, ctypes.byref(inb),
                           None, FAKE, ws, wsz, None)
    assert r == pxm.PX_ERR_INVALID


def pxm_max_parts():
    text = open(os.path.join(ROOT, "include", "px.h")).read()
    return int(re.search(r"#define PX_MAX_PARTS (\d+)", text).group(1))


def test_host_checks_of_later_entry_points(lib):
    import paper_2606_24647_gb300 as pxm
    ws, wsz = FAKE, 1 << 30
    # streaming group-by: unknown flag bits
    g_in = _batch(pxm, [pxm.PX_I32, pxm.PX_I64], 100)
    g_out = _batch(pxm, [pxm.PX_I32, pxm.PX_I64], 100)
    keys = (ctypes.c_int32 * 1)(0)
    aggs = (pxm.px_agg * 1)(pxm.px_agg(pxm.PX_SUM, 1, -1))
    r = lib.px_groupby_agg_stream(ctypes.byref(g_in), keys, 1, aggs, 1, None, None, None, 0, None, 100,
                                  ctypes.byref(g_out), None, FAKE, 8, ws, wsz, None)
    assert r == pxm.PX_ERR_INVALID and "flags" in pxm.last_error()
    # gather: type mismatch between in and out
    gi = _batch(pxm, [pxm.PX_I64], 100)
    go = _batch(pxm, [pxm.PX_I32], 100)
    assert lib.px_gather(ctypes.byref(gi), FAKE, None, ctypes.byref(go), ws, wsz, None) == pxm.PX_ERR_INVALID
    # fused probe + aggregation: key column not int64, null table, no dense range
    p = _batch(pxm, [pxm.PX_I32, pxm.PX_I64], 100)
    grp = pxm.px_col(pxm.PX_I32, 0, FAKE)
    pa = (pxm.px_agg * 1)(pxm.px_agg(pxm.PX_COUNT, -1, -1))
    o = _batch(pxm, [pxm.PX_I32, pxm.PX_I64], 100)
    r = lib.px_join_probe_agg(FAKE, ctypes.byref(p), 0, None, None, None, 0, ctypes.byref(grp), 10, 0, 9, pa, 1,
                              100, ctypes.byref(o), None, FAKE, ws, wsz, None)
    assert r == pxm.PX_ERR_INVALID
    p = _batch(pxm, [pxm.PX_I64, pxm.PX_I64], 100)
    r = lib.px_join_probe_agg(None, ctypes.byref(p), 0, None, None, None, 0, ctypes.byref(grp), 10, 0, 9, pa, 1,
                              100, ctypes.byref(o), None, FAKE, ws, wsz, None)
    assert r == pxm.PX_ERR_INVALID
    r = lib.px_join_probe_agg(FAKE, ctypes.byref(p), 0, None, None, None, 0, ctypes.byref(grp), 10, 0, 1 << 40, pa, 1,
                              100, ctypes.byref(o), None, FAKE, ws, wsz, None)
    assert r == pxm.PX_ERR_UNSUPPORTED
    # fragments: bad configuration, plan staging too small, group range over the limit
    f = (pxm.px_fragment * 1)()
    f[0].nrows = 10
    f[0].key = pxm.px_col(pxm.PX_I64, 0, FAKE)
    f[0].d_table = FAKE
    f[0].nbuild = 10
    f[0].group = pxm.px_col(pxm.PX_I32, 0, FAKE)
    f[0].group_lo, f[0].group_hi = 0, 9
    f[0].max_groups = 10
    f[0].d_out_keys = FAKE
    f[0].d_ngroups = FAKE
    plan = ctypes.create_string_buffer(lib.px_fragments_plan_bytes(1))
    cfg = pxm.px_fragments_config(128, 4, 512, 1)
    assert lib.px_fragments_run(f, 1, ctypes.byref(cfg), plan, len(plan), ws, wsz, None) == pxm.PX_ERR_INVALID
    assert "configuration" in pxm.last_error()
    assert lib.px_fragments_run(f, 1, None, plan, 8, ws, wsz, None) == pxm.PX_ERR_INVALID
    f[0].group_hi = 1 << 23
    assert lib.px_fragments_run(f, 1, None, plan, len(plan), ws, wsz, None) == pxm.PX_ERR_UNSUPPORTED
    # bounded-wait self-test: null pointers and a zero limit
    assert lib.px_selftest_wait(None, 10, FAKE, None) == pxm.PX_ERR_INVALID
    assert lib.px_selftest_wait(FAKE, 0, FAKE, None) == pxm.PX_ERR_INVALID


def test_host_checks_of_join_probe(lib):
    # Every argument error px_join_probe detects on the host, before any GPU work.
    import paper_2606_24647_gb300 as pxm
    ws, wsz = FAKE, 1 << 30
    I32, I64 = pxm.PX_I32, pxm.PX_I64
    probe = _batch(pxm, [I64, I64, I32], 100)
    pay = _batch(pxm, [I32], 50)
    out = _batch(pxm, [I64, I32], 100)
    carry = (ctypes.c_int32 * 1)(1)

    def call(table=FAKE, pb=probe, fk=0, sel=None, nsel=None, seg=None, nsegs=0, cr=carry, ncarry=1, pl=pay,
             ob=out, nout=FAKE, wsb=wsz):
        return lib.px_join_probe(table, ctypes.byref(pb), fk, sel, nsel, seg, nsegs, cr, ncarry,
                                 ctypes.byref(pl) if pl is not None else None, ctypes.byref(ob), None, None, nout,
                                 None, ws, wsb, None)

    cases = [
        (dict(table=None), pxm.PX_ERR_INVALID, "table"),
        (dict(table=FAKE + 8), pxm.PX_ERR_INVALID, "misaligned"),
        (dict(fk=3), pxm.PX_ERR_INVALID, "fk_col"),
        (dict(fk=2), pxm.PX_ERR_INVALID, "PX_I64"),
        (dict(sel=FAKE), pxm.PX_ERR_INVALID, "together"),
        (dict(nsegs=4097, seg=FAKE), pxm.PX_ERR_UNSUPPORTED, "nsegs"),
        (dict(nsegs=4), pxm.PX_ERR_INVALID, "d_seg"),
        (dict(seg=FAKE), pxm.PX_ERR_INVALID, "d_seg"),
        (dict(cr=None), pxm.PX_ERR_INVALID, "carry"),
        (dict(ncarry=-1), pxm.PX_ERR_INVALID, "carry"),
        (dict(pl=None), pxm.PX_ERR_INVALID, "columns"),          # out has one column too many
        (dict(nout=None), pxm.PX_ERR_INVALID, "d_nout"),
        (dict(cr=(ctypes.c_int32 * 1)(7)), pxm.PX_ERR_INVALID, "out of range"),
        (dict(cr=(ctypes.c_int32 * 1)(2)), pxm.PX_ERR_INVALID, "type"),          # carried int32 into int64
        (dict(pl=_batch(pxm, [I64], 50)), pxm.PX_ERR_INVALID, "payload"),       # payload int64 into int32
        (dict(wsb=16), pxm.PX_ERR_INVALID, "px_join_probe"),
    ]
    for kw, want, msg in cases:
        r = call(**kw)
        assert r == want, (kw, r, pxm.last_error())
        assert msg in pxm.last_error(), (kw, pxm.last_error())


def test_host_checks_of_groupby(lib):
    # Every argument error px_groupby_agg detects on the host, before any GPU work.
    import paper_2606_24647_gb300 as pxm
    ws, wsz = FAKE, 1 << 30
    I32, I64 = pxm.PX_I32, pxm.PX_I64
    gin = _batch(pxm, [I32, I64, I64], 100)
    gout = _batch(pxm, [I32, I64, I64], 100)
    one_key = (ctypes.c_int32 * 1)(0)

    def aggs_of(*a):
        return (pxm.px_agg * len(a))(*[pxm.px_agg(*x) for x in a])

    good = aggs_of((pxm.PX_SUM, 1, -1), (pxm.PX_SUM_MUL, 1, 2))

    def call(keys=one_key, nkeys=1, aggs=good, naggs=2, sel=None, nsel=None, seg=None, nsegs=0, max_groups=100,
             ob=gout, ngroups=FAKE, inb=gin, wsb=wsz):
        return lib.px_groupby_agg(ctypes.byref(inb), keys, nkeys, aggs, naggs, sel, nsel, seg, nsegs, None,
                                  max_groups, ctypes.byref(ob), None, ngroups, ws, wsb, None)

    cases = [
        (dict(nkeys=0), pxm.PX_ERR_UNSUPPORTED, "nkeys"),
        (dict(nkeys=3), pxm.PX_ERR_UNSUPPORTED, "nkeys"),
        (dict(naggs=-1), pxm.PX_ERR_UNSUPPORTED, "naggs"),
        (dict(nsel=FAKE), pxm.PX_ERR_INVALID, "together"),
        (dict(nsegs=4097, seg=FAKE), pxm.PX_ERR_UNSUPPORTED, "nsegs"),
        (dict(nsegs=2), pxm.PX_ERR_INVALID, "d_seg"),
        (dict(max_groups=0), pxm.PX_ERR_INVALID, "max_groups"),
        (dict(ngroups=None), pxm.PX_ERR_INVALID, "d_ngroups"),
        (dict(naggs=1), pxm.PX_ERR_INVALID, "columns"),                       # out holds two aggregates
        (dict(max_groups=101), pxm.PX_ERR_INVALID, "capacity"),
        (dict(keys=(ctypes.c_int32 * 1)(5)), pxm.PX_ERR_INVALID, "key column"),
        (dict(keys=(ctypes.c_int32 * 1)(1)), pxm.PX_ERR_INVALID, "type"),     # int64 key into an int32 column
        (dict(aggs=aggs_of((9, 1, -1), (pxm.PX_SUM, 1, -1))), pxm.PX_ERR_INVALID, "unknown op"),
        (dict(aggs=aggs_of((pxm.PX_SUM, 3, -1), (pxm.PX_SUM, 1, -1))), pxm.PX_ERR_INVALID, "column a"),
        (dict(aggs=aggs_of((pxm.PX_SUM, 1, -1), (pxm.PX_SUM_MUL, 1, 7))), pxm.PX_ERR_INVALID, "column b"),
        (dict(ob=_batch(pxm, [I32, I64, I32], 100)), pxm.PX_ERR_INVALID, "PX_I64"),
        (dict(wsb=16), pxm.PX_ERR_INVALID, "px_groupby_agg"),
    ]
    for kw, want, msg in cases:
        r = call(**kw)
        assert r == want, (kw, r, pxm.last_error())
        assert msg in pxm.last_error(), (kw, pxm.last_error())


def test_host_checks_of_join_build_and_gather(lib):
    import paper_2606_24647_gb300 as pxm
    ws, wsz = FAKE, 1 << 30
    I32, I64 = pxm.PX_I32, pxm.PX_I64
    b = _batch(pxm, [I64, I32, I64], 100)
    big = lib.px_join_table_bytes(100, 0)

    def build(bb=b, pk=0, seg=None, nsegs=0, unique=1, pay=-1, table=FAKE, tbytes=1 << 30, wsb=wsz):
        return lib.px_join_build(ctypes.byref(bb), pk, seg, nsegs, unique, pay, table, tbytes, ws, wsb, None)

    cases = [
        (dict(pk=3), pxm.PX_ERR_INVALID, "pk_col"),
        (dict(pay=3), pxm.PX_ERR_INVALID, "pay_col"),
        (dict(pay=0), pxm.PX_ERR_INVALID, "pay_col"),
        (dict(pay=-2), pxm.PX_ERR_INVALID, "pay_col"),
        (dict(pay=2), pxm.PX_ERR_UNSUPPORTED, "PX_I8 or PX_I32"),
        (dict(pk=1), pxm.PX_ERR_INVALID, "PX_I64"),
        (dict(nsegs=4097, seg=FAKE), pxm.PX_ERR_UNSUPPORTED, "nsegs"),
        (dict(nsegs=3), pxm.PX_ERR_INVALID, "d_seg"),
        (dict(seg=FAKE), pxm.PX_ERR_INVALID, "d_seg"),
        (dict(table=None), pxm.PX_ERR_INVALID, "table"),
        (dict(table=FAKE + 4), pxm.PX_ERR_INVALID, "misaligned"),
        (dict(tbytes=big - 1), pxm.PX_ERR_INVALID, "needed"),
        (dict(wsb=16), pxm.PX_ERR_INVALID, "px_join_build"),
    ]
    for kw, want, msg in cases:
        r = build(**kw)
        assert r == want, (kw, r, pxm.last_error())
        assert msg in pxm.last_error(), (kw, pxm.last_error())

    gin = _batch(pxm, [I64, I32], 100)

    def gather(ob, idx=FAKE, wsb=wsz):
        return lib.px_gather(ctypes.byref(gin), idx, None, ctypes.byref(ob), ws, wsb, None)

    assert gather(_batch(pxm, [I64], 10)) == pxm.PX_ERR_INVALID and "columns" in pxm.last_error()
    assert gather(_batch(pxm, [I64, I64], 10)) == pxm.PX_ERR_INVALID and "type" in pxm.last_error()
    assert gather(_batch(pxm, [I64, I32], 10), idx=None) == pxm.PX_ERR_INVALID and "d_idx" in pxm.last_error()
    assert gather(_batch(pxm, [I64, I32], 10), wsb=16) == pxm.PX_ERR_INVALID and "px_gather" in pxm.last_error()
    # no output rows: nothing to do, no index array needed, no GPU work
    assert gather(_batch(pxm, [I64, I32], 0), idx=None) == pxm.PX_OK


def test_binding_refuses_host_tensors():
    # No CPU fallback: a column, pointer or batch built from a host tensor raises
    # before anything reaches the library.
    import torch
    import paper_2606_24647_gb300 as pxm
    host = torch.zeros(16, dtype=torch.int64)
    with pytest.raises(ValueError):
        pxm._col(host)
    with pytest.raises(ValueError):
        pxm._ptr(host)
    with pytest.raises(ValueError):
        pxm._Batch([host])
    with pytest.raises(TypeError):
        pxm._col(torch.zeros(16, dtype=torch.float32))
