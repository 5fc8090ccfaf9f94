"""px: GB300-native hash exchange, hash join and hash aggregation.

Thin ctypes binding of the C ABI in include/px.h (libpx.so, built in-tree by
``paper_2606_24647_gb300.build``). The functions here only marshal arguments:
torch CUDA tensors in, raw device pointers and the caller's CUDA stream out to
the library; every step of the operators runs in the library's CUDA kernels.
There is no CPU fallback: if libpx.so cannot be loaded, or a tensor is not on a
CUDA device, the call raises.

PyTorch is used for device memory (outputs and workspaces are torch tensors) and
streams (``torch.cuda.current_stream()`` unless one is passed).
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpx.so")

PX_OK, PX_ERR_INVALID, PX_ERR_CAPACITY, PX_ERR_DUPLICATE_KEY = 0, 1, 2, 3
PX_ERR_TABLE_FULL, PX_ERR_TIMEOUT, PX_ERR_CUDA, PX_ERR_UNSUPPORTED = 4, 5, 6, 7
STATUS_NAMES = {0: "PX_OK", 1: "PX_ERR_INVALID", 2: "PX_ERR_CAPACITY", 3: "PX_ERR_DUPLICATE_KEY",
                4: "PX_ERR_TABLE_FULL", 5: "PX_ERR_TIMEOUT", 6: "PX_ERR_CUDA", 7: "PX_ERR_UNSUPPORTED"}
PX_I8, PX_I32, PX_I64 = 1, 4, 8
PX_COUNT, PX_SUM, PX_SUM_MUL = 0, 1, 2
PX_AGG_ACCUMULATE, PX_AGG_STREAM = 1, 2

EXPORTED = [
    "px_ws_init", "px_stream_status", "px_last_error", "px_kernel_launches", "px_selftest_wait",
    "px_filter_ws_bytes", "px_filter", "px_filter_noalloc",
    "px_partition_ws_bytes", "px_partition", "px_partition_tuned",
    "px_join_table_bytes", "px_join_build_ws_bytes", "px_join_build",
    "px_join_probe_ws_bytes", "px_join_probe",
    "px_groupby_ws_bytes", "px_groupby_agg", "px_groupby_agg_stream", "px_gather",
    "px_join_probe_agg_ws_bytes", "px_join_probe_agg",
    "px_fragments_plan_bytes", "px_fragments_ws_bytes", "px_fragments_run",
]
PX_FRAG_MAX_COLS, PX_FRAG_MAX_AGGS, PX_FRAG_MAX_GROUPS = 4, 4, 1 << 22

_TYPES = {torch.int8: PX_I8, torch.int32: PX_I32, torch.int64: PX_I64}


class PxError(RuntimeError):
    def __init__(self, status: int, where: str, message: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} {message}".strip())


class px_col(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("reserved", ctypes.c_int32), ("data", ctypes.c_void_p)]


class px_batch(ctypes.Structure):
    _fields_ = [("ncols", ctypes.c_int32), ("reserved", ctypes.c_int32), ("cols", ctypes.POINTER(px_col)),
                ("nrows", ctypes.c_int64), ("d_nrows", ctypes.c_void_p)]


class px_agg(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("a", ctypes.c_int32), ("b", ctypes.c_int32)]


class px_key_range(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int64 * 2), ("hi", ctypes.c_int64 * 2)]


class px_fragment(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("key", px_col), ("filter", px_col), ("lo", ctypes.c_int64),
                ("hi", ctypes.c_int64), ("ncols", ctypes.c_int32), ("naggs", ctypes.c_int32),
                ("cols", px_col * 4), ("aggs", px_agg * 4), ("d_table", ctypes.c_void_p),
                ("nbuild", ctypes.c_int64), ("group", px_col), ("group_lo", ctypes.c_int64),
                ("group_hi", ctypes.c_int64), ("max_groups", ctypes.c_int64), ("d_out_keys", ctypes.c_void_p),
                ("d_out_aggs", ctypes.c_void_p * 4), ("d_ngroups", ctypes.c_void_p)]


class px_partition_config(ctypes.Structure):
    _fields_ = [("items", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32)]


class px_fragments_config(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("items", ctypes.c_int32), ("chunk_rows", ctypes.c_int64),
                ("blocks_per_sm", ctypes.c_int32)]


_lib = None


def _declare(lib):
    P, I32, I64, U64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
    BP = ctypes.POINTER(px_batch)
    CP = ctypes.POINTER(px_col)
    AP = ctypes.POINTER(px_agg)
    sig = {
        "px_ws_init": ([P, SZ, P], I32),
        "px_stream_status": ([P, P], I32),
        "px_last_error": ([], ctypes.c_char_p),
        "px_kernel_launches": ([], U64),
        "px_selftest_wait": ([P, ctypes.c_uint32, P, P], I32),
        "px_filter_ws_bytes": ([I64], SZ),
        "px_filter": ([CP, I64, P, I64, I64, P, P, P, SZ, P], I32),
        "px_filter_noalloc": ([CP, I64, P, I64, I64, P, P, P, P], I32),
        "px_partition_ws_bytes": ([I64, I32], SZ),
        "px_partition": ([BP, I32, P, P, I32, U64, BP, P, P, SZ, P], I32),
        "px_partition_tuned": ([BP, I32, P, P, I32, U64, BP, P, ctypes.POINTER(px_partition_config), P, SZ, P], I32),
        "px_join_table_bytes": ([I64, I32], SZ),
        "px_join_build_ws_bytes": ([I64], SZ),
        "px_join_build": ([BP, I32, P, I32, I32, I32, P, SZ, P, SZ, P], I32),
        "px_join_probe_ws_bytes": ([I64], SZ),
        "px_join_probe": ([P, BP, I32, P, P, P, I32, P, I32, BP, BP, P, P, P, P, P, SZ, P], I32),
        "px_groupby_ws_bytes": ([I64, I64], SZ),
        "px_groupby_agg": ([BP, P, I32, AP, I32, P, P, P, I32, ctypes.POINTER(px_key_range), I64, BP, P, P, P,
                            SZ, P], I32),
        "px_groupby_agg_stream": ([BP, P, I32, AP, I32, P, P, P, I32, ctypes.POINTER(px_key_range), I64, BP, P, P,
                                   I32, P, SZ, P], I32),
        "px_gather": ([BP, P, P, BP, P, SZ, P], I32),
        "px_join_probe_agg_ws_bytes": ([I64, I64], SZ),
        "px_join_probe_agg": ([P, BP, I32, P, P, P, I32, CP, I64, I64, I64, AP, I32, I64, BP, P, P, P, SZ, P], I32),
        "px_fragments_plan_bytes": ([I32], SZ),
        "px_fragments_ws_bytes": ([ctypes.POINTER(px_fragment), I32], SZ),
        "px_fragments_run": ([ctypes.POINTER(px_fragment), I32, ctypes.POINTER(px_fragments_config), P, SZ, P, SZ, P],
                             I32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res


def load(path: str | None = None):
    """Load libpx.so (building it first if its sources are newer). Raises if it is missing."""
    global _lib
    if _lib is None:
        from . import build as _build
        if path is None:
            if _build.stale() and os.path.exists(_build.NVCC):
                _build.build()
            path = LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(f"px CUDA library not found at {path}; run paper_2606_24647_gb300.build.build()")
        lib = ctypes.CDLL(path)
        _declare(lib)
        _lib = lib
    return _lib


def lib():
    return load()


def last_error() -> str:
    return (load().px_last_error() or b"").decode()


def kernel_launches() -> int:
    """Kernels launched by libpx.so in this process so far."""
    return int(load().px_kernel_launches())


def _check(status: int, where: str):
    if status != PX_OK:
        raise PxError(status, where, last_error())


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("px tensors must be CUDA tensors")
    return t.data_ptr()


def _sel_ptr(sel) -> int | None:
    """Device pointer of a selection vector; an empty one (null data in torch) is
    replaced by a one-element buffer, its device count still says zero rows."""
    if sel is not None and sel.numel() == 0:
        sel = torch.zeros(1, dtype=torch.int32, device=sel.device)
        _keep_alive.append(sel)
        del _keep_alive[:-8]
    return _ptr(sel)


_keep_alive: list = []


def _stream(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _col(t: torch.Tensor) -> px_col:
    if t.dtype not in _TYPES:
        raise TypeError(f"unsupported column dtype {t.dtype}")
    if not t.is_cuda or not t.is_contiguous() or t.dim() != 1:
        raise ValueError("columns must be contiguous 1-D CUDA tensors")
    return px_col(_TYPES[t.dtype], 0, t.data_ptr())


class _Batch:
    """A px_batch plus the ctypes storage it points into."""

    def __init__(self, cols, nrows=None, d_nrows=None):
        self.cols = list(cols)
        self.arr = (px_col * max(1, len(self.cols)))(*[_col(c) for c in self.cols])
        n = nrows if nrows is not None else (self.cols[0].numel() if self.cols else 0)
        self.b = px_batch(len(self.cols), 0, ctypes.cast(self.arr, ctypes.POINTER(px_col)), n, _ptr(d_nrows))

    def ref(self):
        return ctypes.byref(self.b)


class Workspace:
    """Caller-owned device workspace (a torch uint8 tensor), grown on demand.

    The first 256 bytes hold the sticky status word; px_ws_init clears them."""

    def __init__(self, nbytes: int = 1 << 20, device=None, stream=None):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.buf = torch.zeros(max(nbytes, 256), dtype=torch.uint8, device=self.device)

    def ensure(self, nbytes: int, stream=None):
        if self.buf.numel() < nbytes:
            self.buf = torch.zeros(int(nbytes * 1.25) + 256, dtype=torch.uint8, device=self.device)
        return self

    @property
    def ptr(self) -> int:
        return self.buf.data_ptr()

    @property
    def nbytes(self) -> int:
        return self.buf.numel()

    def reset(self, stream=None):
        _check(load().px_ws_init(self.ptr, self.nbytes, _stream(stream)), "px_ws_init")

    def status(self, stream=None) -> int:
        return int(load().px_stream_status(_stream(stream), self.ptr))


def _ws(ws, need, stream):
    if ws is None:
        ws = Workspace(need)
    ws.ensure(need, stream)
    return ws


def px_stream_status(ws: Workspace, stream=None) -> int:
    """Synchronise the stream and return the workspace's sticky status word."""
    return ws.status(stream)


def px_ws_init(ws: Workspace, stream=None):
    ws.reset(stream)


def px_filter(col, lo: int, hi: int, *, d_nrows=None, sel=None, nsel=None, ws=None, stream=None):
    """Selection of rows with lo <= col < hi (FilterProject, Sec. 3.2). Returns (sel, nsel)."""
    L = load()
    n = col.numel()
    sel = sel if sel is not None else torch.empty(max(n, 1), dtype=torch.int32, device=col.device)
    nsel = nsel if nsel is not None else torch.empty(1, dtype=torch.int64, device=col.device)
    ws = _ws(ws, L.px_filter_ws_bytes(n), stream)
    c = _col(col)
    _check(L.px_filter(ctypes.byref(c), n, _ptr(d_nrows), int(lo), int(hi), _ptr(sel), _ptr(nsel),
                       ws.ptr, ws.nbytes, _stream(stream)), "px_filter")
    return sel, nsel


def px_partition(cols, key_col: int, nparts: int, seed: int = 0, *, sel=None, nsel=None, d_nrows=None,
                 out=None, offsets=None, config=None, ws=None, stream=None):
    """Hash repartition into nparts stable segments (the exchange, Sec. 3.1/3.3.2).
    config: optional (items, blocks_per_sm) launch shape (px_partition_tuned).

    Returns (out_cols, offsets int64[nparts+1])."""
    L = load()
    n = cols[0].numel()
    inb = _Batch(cols, n, d_nrows)
    out = out if out is not None else [torch.empty(max(n, 1), dtype=c.dtype, device=c.device) for c in cols]
    outb = _Batch(out, max(n, 1))
    offsets = offsets if offsets is not None else torch.empty(nparts + 1, dtype=torch.int64, device=cols[0].device)
    ws = _ws(ws, L.px_partition_ws_bytes(n, nparts), stream)
    if config is None:
        _check(L.px_partition(inb.ref(), key_col, _sel_ptr(sel), _ptr(nsel), nparts, int(seed) & (2**64 - 1),
                              outb.ref(), _ptr(offsets), ws.ptr, ws.nbytes, _stream(stream)), "px_partition")
    else:
        cfg = px_partition_config(*config)
        _check(L.px_partition_tuned(inb.ref(), key_col, _sel_ptr(sel), _ptr(nsel), nparts, int(seed) & (2**64 - 1),
                                    outb.ref(), _ptr(offsets), ctypes.byref(cfg), ws.ptr, ws.nbytes,
                                    _stream(stream)), "px_partition")
    return out, offsets


def px_join_build(cols, pk_col: int, *, seg=None, unique: bool = True, pay_col=None, d_nrows=None, table=None,
                  ws=None, stream=None):
    """Build a (per-segment) hash table on cols[pk_col] (join build pipeline). Returns the table tensor.

    pay_col: a build column (int8 or int32) copied beside each key; probes whose payload
    is exactly that column read the copy instead of gathering it."""
    L = load()
    n = cols[0].numel()
    nsegs = 0 if seg is None else seg.numel() - 1
    need = L.px_join_table_bytes(n, nsegs)
    table = table if table is not None and table.numel() >= need else torch.empty(
        need, dtype=torch.uint8, device=cols[0].device)
    b = _Batch(cols, n, d_nrows)
    ws = _ws(ws, L.px_join_build_ws_bytes(n), stream)
    _check(L.px_join_build(b.ref(), pk_col, _ptr(seg), nsegs, 1 if unique else 0, -1 if pay_col is None else pay_col,
                           table.data_ptr(), table.numel(), ws.ptr, ws.nbytes, _stream(stream)), "px_join_build")
    return table


def px_join_probe(table, cols, fk_col: int, *, sel=None, nsel=None, seg=None, d_nrows=None, carry=(),
                  payload=None, out_cap=None, out=None, probe_row=False, build_row=False, out_seg=False,
                  ws=None, stream=None):
    """Inner equi-join probe (join probe pipeline). Returns a dict with 'cols' (carried probe
    columns then payload columns), 'nout' (device int64[1]) and optionally 'probe_row',
    'build_row' (int32) and 'out_seg' (int64[nsegs+1])."""
    L = load()
    n = cols[0].numel()
    dev = cols[0].device
    nsegs = 0 if seg is None else seg.numel() - 1
    cap = out_cap if out_cap is not None else max(n, 1)
    carry = list(carry)
    pay = list(payload) if payload is not None else []
    if out is None:
        out = [torch.empty(cap, dtype=cols[c].dtype, device=dev) for c in carry] + \
              [torch.empty(cap, dtype=p.dtype, device=dev) for p in pay]
    pb = _Batch(cols, n, d_nrows)
    payb = _Batch(pay) if pay else None
    outb = _Batch(out, cap)
    res = {"cols": out, "nout": torch.empty(1, dtype=torch.int64, device=dev)}
    if probe_row:
        res["probe_row"] = torch.empty(cap, dtype=torch.int32, device=dev)
    if build_row:
        res["build_row"] = torch.empty(cap, dtype=torch.int32, device=dev)
    if out_seg:
        res["out_seg"] = torch.empty(max(nsegs, 1) + 1, dtype=torch.int64, device=dev)
    carr = (ctypes.c_int32 * max(1, len(carry)))(*carry)
    ws = _ws(ws, L.px_join_probe_ws_bytes(n), stream)
    _check(L.px_join_probe(table.data_ptr(), pb.ref(), fk_col, _sel_ptr(sel), _ptr(nsel), _ptr(seg), nsegs,
                           carr, len(carry), payb.ref() if payb else None, outb.ref(),
                           _ptr(res.get("probe_row")), _ptr(res.get("build_row")), _ptr(res["nout"]),
                           _ptr(res.get("out_seg")), ws.ptr, ws.nbytes, _stream(stream)), "px_join_probe")
    return res


def px_groupby_agg(cols, key_cols, aggs, *, max_groups: int, sel=None, nsel=None, seg=None, d_nrows=None,
                   key_range=None, out=None, ws=None, stream=None, flags: int = 0, ngroups=None, out_seg=None):
    """GROUP BY key_cols computing aggs = [(op, a, b), ...] (HashAggregation, Sec. 3.2).

    key_range: optional [(lo, hi), ...] per key column, a statistic of where the keys
    lie (speed only; rows outside are still aggregated exactly).
    Returns a dict with 'keys' (list of key columns), 'aggs' (list of int64 columns),
    'seg' (int32 segment per group when segmented) and 'ngroups' (device int64[1]); the
    first ngroups rows are valid, in unspecified order."""
    L = load()
    n = cols[0].numel()
    dev = cols[0].device
    nsegs = 0 if seg is None else seg.numel() - 1
    if out is None:
        out = [torch.empty(max_groups, dtype=cols[k].dtype, device=dev) for k in key_cols] + \
              [torch.empty(max_groups, dtype=torch.int64, device=dev) for _ in aggs]
    inb = _Batch(cols, n, d_nrows)
    outb = _Batch(out, max_groups)
    karr = (ctypes.c_int32 * len(key_cols))(*key_cols)
    aarr = (px_agg * max(1, len(aggs)))(*[px_agg(op, a if a is not None else -1, b if b is not None else -1)
                                          for op, a, b in aggs])
    res = {"keys": out[:len(key_cols)], "aggs": out[len(key_cols):],
           "ngroups": ngroups if ngroups is not None else torch.empty(1, dtype=torch.int64, device=dev)}
    if nsegs > 0:
        res["seg"] = out_seg if out_seg is not None else torch.empty(max_groups, dtype=torch.int32, device=dev)
    rng = None
    if key_range is not None:
        rng = px_key_range()
        for k, (lo, hi) in enumerate(key_range):
            rng.lo[k], rng.hi[k] = int(lo), int(hi)
    ws = _ws(ws, L.px_groupby_ws_bytes(n, max_groups), stream)
    args = (inb.ref(), karr, len(key_cols), aarr, len(aggs), _sel_ptr(sel), _ptr(nsel), _ptr(seg), nsegs,
            ctypes.byref(rng) if rng is not None else None, max_groups, outb.ref(), _ptr(res.get("seg")),
            _ptr(res["ngroups"]))
    if flags:
        _check(L.px_groupby_agg_stream(*args, int(flags), ws.ptr, ws.nbytes, _stream(stream)), "px_groupby_agg_stream")
    else:
        _check(L.px_groupby_agg(*args, ws.ptr, ws.nbytes, _stream(stream)), "px_groupby_agg")
    return res


def fragment_descriptor(f: dict) -> tuple:
    """The px_fragment descriptor of one fragment dict (see FragmentBatch), its
    result tensors {'keys', 'aggs', 'ngroups'} (the dict's 'out' = (keys, [aggs],
    ngroups) when given, else allocated here) and the tensors the descriptor points
    to (kept alive with it)."""
    d = px_fragment()
    key = f["key"]
    dev = key.device
    d.nrows = key.numel()
    d.key = _col(key)
    if f.get("filter") is not None:
        d.filter = _col(f["filter"])
        d.lo, d.hi = int(f["lo"]), int(f["hi"])
    cols = list(f.get("cols", []))
    d.ncols = len(cols)
    for c, t in enumerate(cols):
        d.cols[c] = _col(t)
    aggs = list(f.get("aggs", []))
    d.naggs = len(aggs)
    for a, (op, x, y) in enumerate(aggs):
        d.aggs[a] = px_agg(op, -1 if x is None else x, -1 if y is None else y)
    d.d_table = _ptr(f["table"])
    d.nbuild = f["group"].numel()
    d.group = _col(f["group"])
    d.group_lo, d.group_hi = int(f["group_lo"]), int(f["group_hi"])
    mg = int(f["max_groups"])
    d.max_groups = mg
    if f.get("out") is not None:  # caller-provided outputs: (keys, [aggs...], ngroups)
        keys, outs, ng = f["out"][0], list(f["out"][1]), f["out"][2]
    else:
        keys = torch.empty(max(mg, 1), dtype=f["group"].dtype, device=dev)
        outs = [torch.empty(max(mg, 1), dtype=torch.int64, device=dev) for _ in aggs]
        ng = torch.zeros(1, dtype=torch.int64, device=dev)
    d.d_out_keys = keys.data_ptr()
    for a, t in enumerate(outs):
        d.d_out_aggs[a] = t.data_ptr()
    d.d_ngroups = ng.data_ptr()
    return d, {"keys": keys, "aggs": outs, "ngroups": ng}, [key, f.get("filter"), f["table"], f["group"], *cols]


class FragmentBatch:
    """A batch of fused filter -> join probe -> aggregate fragments (px_fragments_run).

    Each fragment is a dict with: key (int64 probe join-key column), filter (column
    or None), lo, hi (keep lo <= filter < hi), cols (probe columns the aggregates
    read), aggs [(op, a, b)], table (a unique unsegmented table from px_join_build),
    group (build column holding the group key, indexed by build row), group_lo,
    group_hi (every group key lies in that range) and max_groups. Outputs are
    allocated once; run() may be called again (one run in flight per batch). The
    pinned plan staging buffer lives with the batch."""

    def __init__(self, frags: list, config: tuple | None = None, ws: Workspace | None = None,
                 plan: torch.Tensor | None = None, prepared: list | None = None):
        """frags: fragment dicts; or prepared: (descriptor, results, tensors) triples
        from fragment_descriptor, built once per fragment and reused across batches
        (a serving loop forms a batch by copying descriptors only)."""
        L = load()
        if prepared is None:
            prepared = [fragment_descriptor(f) for f in frags]
        self.n = len(prepared)
        self.frags = frags
        arr = (px_fragment * max(1, self.n))()
        for i, (d, _, _) in enumerate(prepared):
            arr[i] = d
        self.results = [r for _, r, _ in prepared]
        self._keep = [k for _, _, k in prepared]
        dev = self.results[0]["keys"].device if prepared else torch.device("cuda", torch.cuda.current_device())
        self.arr = arr
        self.cfg = None
        if config is not None:
            self.cfg = px_fragments_config(*config)
        pb = max(1, L.px_fragments_plan_bytes(self.n))
        self.plan = plan if plan is not None and plan.numel() >= pb else torch.empty(pb, dtype=torch.uint8).pin_memory()
        need = L.px_fragments_ws_bytes(arr, self.n)
        self.ws = (ws or Workspace(need, device=dev)).ensure(need)

    def run(self, stream=None, config: tuple | None = None):
        """Launch the batch (config overrides the batch's launch configuration)."""
        L = load()
        cfg = px_fragments_config(*config) if config is not None else self.cfg
        _check(L.px_fragments_run(self.arr, self.n, ctypes.byref(cfg) if cfg is not None else None,
                                  self.plan.data_ptr(), self.plan.numel(), self.ws.ptr, self.ws.nbytes,
                                  _stream(stream)), "px_fragments_run")
        return self.results


def px_selftest_wait(flag: torch.Tensor, spin_limit: int, status: torch.Tensor, stream=None) -> None:
    """Bounded device wait on flag (int32[1]) -> status (int32[1]): PX_OK or PX_ERR_TIMEOUT."""
    _check(load().px_selftest_wait(_ptr(flag), int(spin_limit), _ptr(status), _stream(stream)), "px_selftest_wait")


def px_gather(cols, idx, *, n=None, d_n=None, out=None, ws=None, stream=None):
    """out[c][i] = cols[c][idx[i]] for the first n positions (or *d_n) - the gather of
    late materialization. Returns the output columns."""
    L = load()
    cap = idx.numel() if n is None else int(n)
    dev = idx.device
    if out is None:
        out = [torch.empty(max(cap, 1), dtype=c.dtype, device=dev) for c in cols]
    inb = _Batch(cols, cols[0].numel(), None)
    outb = _Batch(out, cap)
    ws = _ws(ws, 256, stream)
    _check(L.px_gather(inb.ref(), _ptr(idx), _ptr(d_n), outb.ref(), ws.ptr, ws.nbytes, _stream(stream)), "px_gather")
    return out


def px_join_probe_agg(table, cols, fk_col: int, group, group_range, aggs, *, max_groups: int, sel=None, nsel=None,
                      seg=None, d_nrows=None, out=None, ngroups=None, out_seg=None, ws=None, stream=None):
    """Join probe fused with the aggregation grouping by the build column `group`
    (values in group_range = (lo, hi)); aggs index the probe columns. Returns a dict
    like px_groupby_agg's ('keys', 'aggs', 'ngroups', 'seg' when segmented)."""
    L = load()
    n = cols[0].numel()
    dev = cols[0].device
    nsegs = 0 if seg is None else seg.numel() - 1
    if out is None:
        out = [torch.empty(max_groups, dtype=group.dtype, device=dev)] + \
              [torch.empty(max_groups, dtype=torch.int64, device=dev) for _ in aggs]
    inb = _Batch(cols, n, d_nrows)
    outb = _Batch(out, max_groups)
    aarr = (px_agg * max(1, len(aggs)))(*[px_agg(op, a if a is not None else -1, b if b is not None else -1)
                                          for op, a, b in aggs])
    g = _col(group)
    res = {"keys": out[:1], "aggs": out[1:],
           "ngroups": ngroups if ngroups is not None else torch.empty(1, dtype=torch.int64, device=dev)}
    if nsegs > 0:
        res["seg"] = out_seg if out_seg is not None else torch.empty(max_groups, dtype=torch.int32, device=dev)
    ws = _ws(ws, L.px_join_probe_agg_ws_bytes(n, max_groups), stream)
    _check(L.px_join_probe_agg(_ptr(table), inb.ref(), fk_col, _sel_ptr(sel), _ptr(nsel), _ptr(seg), nsegs,
                               ctypes.byref(g), group.numel(), int(group_range[0]), int(group_range[1]), aarr,
                               len(aggs), max_groups, outb.ref(), _ptr(res.get("seg")), _ptr(res["ngroups"]),
                               ws.ptr, ws.nbytes, _stream(stream)), "px_join_probe_agg")
    return res
