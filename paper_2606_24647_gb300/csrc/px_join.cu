// px_join_build / px_join_probe: the join build and probe pipelines (Sec. 3.1;
// the join-heavy queries Q5/Q9 of Sec. 3.4), per partition after the exchange
// when segments are given.
//
// Table (caller memory, private layout):
//   [0, 64)            header: magic, nsegs, unique flag
//   [64, 64 + A)       copy of the build segment offsets (nsegs + 1 int64)
//   [64 + A, ...)      slots of 16 bytes {int64 key, int32 build row, int32 pad}
// Segment q of n_q rows owns 2 n_q + 2 slots starting at slot 2 seg[q] + 2 q, so
// every segment runs at load factor <= 1/2 and the whole table is exactly
// 2 n + 2 nsegs slots with no size known before the build. A key's home slot is
// the multiply-shift reduction of the LOWER 32 bits of fmix64(key) (the exchange
// uses the upper 32), then linear probing. Empty slots hold INT64_MIN.
#include <algorithm>

#include "px_common.cuh"

namespace px {
namespace {

constexpr int64_t kEmpty = INT64_MIN;
constexpr int64_t kMagic = 0x707874626c763031ll;  // "pxtblv01"

struct TableHeader {
    int64_t magic;
    int32_t nsegs;   // >= 1
    int32_t unique;
    int64_t nbuild;  // build rows inserted
    int64_t reserved[5];
};

struct Slot {
    int64_t key;
    int32_t row;
    int32_t pad;
};

size_t seg_area_bytes(int32_t S) { return align_up(static_cast<size_t>(S + 1) * 8, 64); }

struct TableView {
    TableHeader* hdr;
    int64_t* seg;
    Slot* slots;
};

TableView table_view(void* d_table, int32_t S) {
    TableView t;
    char* b = static_cast<char*>(d_table);
    t.hdr = reinterpret_cast<TableHeader*>(b);
    t.seg = reinterpret_cast<int64_t*>(b + 64);
    t.slots = reinterpret_cast<Slot*>(b + 64 + seg_area_bytes(S));
    return t;
}

// ------------------------------------------------------------------ build ----

__global__ void build_init_kernel(TableView t, int32_t S, int32_t unique, const int64_t* __restrict__ d_seg,
                                  const int64_t* __restrict__ d_n, int64_t ncap) {
    const int64_t n = actual_rows(d_n, ncap);
    const int64_t gtid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    if (gtid == 0) {
        t.hdr->magic = kMagic;
        t.hdr->nsegs = S;
        t.hdr->unique = unique;
        t.hdr->nbuild = n;
        // Segment offsets clamped to be non-decreasing within [0, n] and to end at
        // n, so no segment can address a slot outside the table.
        int64_t prev = 0;
        t.seg[0] = 0;
        for (int q = 1; q < S; ++q) {
            int64_t v = d_seg ? d_seg[q] : n;
            v = v < prev ? prev : (v > n ? n : v);
            t.seg[q] = v;
            prev = v;
        }
        t.seg[S] = n;
    }
    const int64_t nslots = 2 * n + 2 * static_cast<int64_t>(S);
    longlong2* s2 = reinterpret_cast<longlong2*>(t.slots);
    for (int64_t s = gtid; s < nslots; s += stride) s2[s] = make_longlong2(kEmpty, 0xffffffffll);
}

__global__ void build_insert_kernel(TableView t, int32_t S, int32_t unique, const int64_t* __restrict__ pk,
                                    const int64_t* __restrict__ d_n, int64_t ncap, int32_t* status) {
    const int64_t n = actual_rows(d_n, ncap);
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t key = pk[i];
    if (key == kEmpty) {
        set_status(status, PX_ERR_UNSUPPORTED);
        return;
    }
    const int q = S > 1 ? seg_of(t.seg, S, i) : 0;
    const int64_t s0 = t.seg[q], s1 = t.seg[q + 1];
    const int64_t base = 2 * s0 + 2 * static_cast<int64_t>(q);
    const uint32_t cap = static_cast<uint32_t>(2 * (s1 - s0) + 2);
    uint32_t s = slot_of(fmix64(static_cast<uint64_t>(key)), cap);
    for (uint32_t probe = 0; probe < cap; ++probe) {
        Slot* slot = &t.slots[base + s];
        const unsigned long long prev = atomicCAS(reinterpret_cast<unsigned long long*>(&slot->key),
                                                  static_cast<unsigned long long>(kEmpty),
                                                  static_cast<unsigned long long>(key));
        if (prev == static_cast<unsigned long long>(kEmpty)) {
            slot->row = static_cast<int32_t>(i);
            return;
        }
        if (unique && prev == static_cast<unsigned long long>(key)) {
            set_status(status, PX_ERR_DUPLICATE_KEY);
            return;
        }
        if (++s == cap) s = 0;
    }
    set_status(status, PX_ERR_TABLE_FULL);
}

// ------------------------------------------------------------------ probe ----

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;
constexpr int kWarps = kThreads / 32;

struct OutCols {
    int32_t ncarry, npay;
    int32_t carry_w[PX_MAX_COLS];
    const void* carry_in[PX_MAX_COLS];
    void* carry_out[PX_MAX_COLS];
    int32_t pay_w[PX_MAX_COLS];
    const void* pay_in[PX_MAX_COLS];
    void* pay_out[PX_MAX_COLS];
};

__device__ __forceinline__ void copy_cell(void* out, const void* in, int w, int64_t dst, int64_t src) {
    if (w == 8) static_cast<int64_t*>(out)[dst] = static_cast<const int64_t*>(in)[src];
    else if (w == 4) static_cast<int32_t*>(out)[dst] = static_cast<const int32_t*>(in)[src];
    else static_cast<int8_t*>(out)[dst] = static_cast<const int8_t*>(in)[src];
}

__device__ __forceinline__ void emit(const OutCols& oc, int64_t pos, int64_t prow, int64_t brow,
                                     int32_t* probe_row, int32_t* build_row) {
    if (probe_row) probe_row[pos] = static_cast<int32_t>(prow);
    if (build_row) build_row[pos] = static_cast<int32_t>(brow);
    for (int c = 0; c < oc.ncarry; ++c) copy_cell(oc.carry_out[c], oc.carry_in[c], oc.carry_w[c], pos, prow);
    for (int c = 0; c < oc.npay; ++c) copy_cell(oc.pay_out[c], oc.pay_in[c], oc.pay_w[c], pos, brow);
}

__global__ void __launch_bounds__(kThreads)
probe_kernel(TableView t, int32_t S, const int64_t* __restrict__ fk, const int32_t* __restrict__ sel,
             const int64_t* __restrict__ d_n, int64_t ncap, const int64_t* __restrict__ pseg, OutCols oc,
             int32_t* __restrict__ probe_row, int32_t* __restrict__ build_row, int64_t out_cap,
             int64_t* __restrict__ d_nout, int64_t* __restrict__ d_out_seg, ScanScratch scan, int32_t* status,
             int64_t ntiles, int64_t payload_rows) {
    __shared__ int64_t s_tile;
    __shared__ int64_t s_excl;
    __shared__ int32_t s_warp[kWarps];
    __shared__ int32_t s_bad;
    const int64_t tile = next_tile(scan.counter, &s_tile);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0)
        s_bad = (t.hdr->magic != kMagic || t.hdr->nsegs != S || (oc.npay > 0 && t.hdr->nbuild > payload_rows)) ? 1 : 0;
    const int64_t n = actual_rows(d_n, ncap);
    const bool unique = t.hdr->unique != 0;
    const int64_t base = tile * kTile + warp * (32 * kItems);
    __syncthreads();
    const bool bad = s_bad != 0;
    if (bad && threadIdx.x == 0) set_status(status, PX_ERR_INVALID);

    int32_t m[kItems];      // matches of this position
    int32_t first[kItems];  // slot (within segment) of the first match
    int32_t brow[kItems];   // build row of the first match
    int32_t prow[kItems];
    int32_t segq[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int64_t j = base + i * 32 + lane;
        m[i] = 0;
        first[i] = 0;
        brow[i] = -1;
        prow[i] = 0;
        segq[i] = 0;
        if (j < n && !bad) {
            const int64_t r = sel ? static_cast<int64_t>(sel[j]) : j;
            prow[i] = static_cast<int32_t>(r);
            const int64_t key = fk[r];
            const int q = S > 1 ? seg_of(pseg, S, j) : 0;
            segq[i] = q;
            if (key == kEmpty) continue;
            const int64_t s0 = t.seg[q], s1 = t.seg[q + 1];
            const Slot* seg_slots = t.slots + 2 * s0 + 2 * static_cast<int64_t>(q);
            const uint32_t cap = static_cast<uint32_t>(2 * (s1 - s0) + 2);
            uint32_t s = slot_of(fmix64(static_cast<uint64_t>(key)), cap);
            for (uint32_t probe = 0; probe < cap; ++probe) {
                const longlong2 v = *reinterpret_cast<const longlong2*>(&seg_slots[s]);
                if (v.x == key) {
                    if (m[i] == 0) {
                        first[i] = static_cast<int32_t>(s);
                        brow[i] = static_cast<int32_t>(v.y);
                    }
                    ++m[i];
                    if (unique) break;
                } else if (v.x == kEmpty) {
                    break;
                }
                if (++s == cap) s = 0;
            }
        }
    }
    // Exclusive output offsets in position order (warp, item, lane).
    int32_t pre[kItems];
    int32_t wsum = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int32_t incl = warp_incl_scan(m[i]);
        pre[i] = wsum + incl - m[i];
        wsum += __shfl_sync(FULL, incl, 31);
    }
    if (lane == 0) s_warp[warp] = wsum;
    __syncthreads();
    if (warp == 0) {
        const int32_t w = lane < kWarps ? s_warp[lane] : 0;
        const int32_t incl = warp_incl_scan(w);
        const int32_t total = __shfl_sync(FULL, incl, 31);
        if (lane < kWarps) s_warp[lane] = incl - w;
        const int64_t excl = lookback(scan.states, tile, total, status);
        if (lane == 0) {
            s_excl = excl;
            if (tile == ntiles - 1) {
                *d_nout = excl + total;
                if (excl + total > out_cap) set_status(status, PX_ERR_CAPACITY);
            }
        }
    }
    __syncthreads();
    const int64_t wbase = s_excl + s_warp[warp];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int64_t j = base + i * 32 + lane;
        const int64_t pos0 = wbase + pre[i];
        if (d_out_seg && j < n) {
            for (int q = segq[i]; q >= 0 && (S > 1 ? pseg[q] == j : j == 0); --q) d_out_seg[q] = pos0;
        }
        if (m[i] == 0) continue;
        if (unique || m[i] == 1) {
            if (pos0 < out_cap) emit(oc, pos0, prow[i], brow[i], probe_row, build_row);
            continue;
        }
        // Multi-match: walk the probe sequence again from the first match.
        const int q = segq[i];
        const int64_t s0 = t.seg[q], s1 = t.seg[q + 1];
        const Slot* seg_slots = t.slots + 2 * s0 + 2 * static_cast<int64_t>(q);
        const uint32_t cap = static_cast<uint32_t>(2 * (s1 - s0) + 2);
        const int64_t key = fk[prow[i]];
        uint32_t s = static_cast<uint32_t>(first[i]);
        int64_t pos = pos0;
        for (uint32_t probe = 0; probe < cap && pos < pos0 + m[i]; ++probe) {
            const longlong2 v = *reinterpret_cast<const longlong2*>(&seg_slots[s]);
            if (v.x == key) {
                if (pos < out_cap) emit(oc, pos, prow[i], static_cast<int32_t>(v.y), probe_row, build_row);
                ++pos;
            } else if (v.x == kEmpty) {
                break;
            }
            if (++s == cap) s = 0;
        }
    }
}

// Segment starts at or past the end of the positions: out_seg[q] = nout.
__global__ void probe_seg_tail_kernel(const int64_t* __restrict__ pseg, int32_t S, int32_t segmented,
                                      const int64_t* __restrict__ d_n, int64_t ncap, const int64_t* __restrict__ d_nout,
                                      int64_t* __restrict__ d_out_seg) {
    const int64_t n = actual_rows(d_n, ncap);
    for (int q = threadIdx.x; q <= S; q += blockDim.x) {
        const int64_t start = segmented ? pseg[q] : (q == 0 ? 0 : n);
        if (start >= n) d_out_seg[q] = *d_nout;
    }
}

}  // namespace
}  // namespace px

using namespace px;

extern "C" {

size_t px_join_table_bytes(int64_t nbuild, int32_t nsegs) {
    if (nbuild < 0) nbuild = 0;
    const int32_t S = nsegs > 0 ? nsegs : 1;
    return 64 + seg_area_bytes(S) + (2 * static_cast<size_t>(nbuild) + 2 * static_cast<size_t>(S)) * sizeof(Slot);
}

size_t px_join_build_ws_bytes(int64_t nbuild) {
    (void)nbuild;
    return kWsScratch;
}

size_t px_join_probe_ws_bytes(int64_t nprobe) {
    if (nprobe < 0) nprobe = 0;
    return kWsScratch + scan_scratch_bytes(cdiv(nprobe, kTile));
}

px_status px_join_build(const px_batch* build, int32_t pk_col, const int64_t* d_seg, int32_t nsegs, int32_t unique,
                        void* d_table, size_t table_bytes, void* d_ws, size_t ws_bytes, void* stream) {
    set_error("");
    px_status s = check_batch(build, "px_join_build build");
    if (s != PX_OK) return s;
    if (pk_col < 0 || pk_col >= build->ncols) return fail(PX_ERR_INVALID, "px_join_build: pk_col %d", pk_col);
    if (build->cols[pk_col].type != PX_I64) return fail(PX_ERR_INVALID, "px_join_build: key column must be PX_I64");
    if (nsegs < 0 || nsegs > PX_MAX_SEGS)
        return fail(PX_ERR_UNSUPPORTED, "px_join_build: nsegs %d outside [0, %d]", nsegs, PX_MAX_SEGS);
    if ((nsegs > 0) != (d_seg != nullptr))
        return fail(PX_ERR_INVALID, "px_join_build: d_seg must be given exactly when nsegs > 0");
    if (!d_table || !aligned16(d_table)) return fail(PX_ERR_INVALID, "px_join_build: null or misaligned table");
    if (table_bytes < px_join_table_bytes(build->nrows, nsegs))
        return fail(PX_ERR_INVALID, "px_join_build: table of %zu bytes, %zu needed", table_bytes,
                    px_join_table_bytes(build->nrows, nsegs));
    s = check_ws(d_ws, ws_bytes, px_join_build_ws_bytes(build->nrows), "px_join_build");
    if (s != PX_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int32_t S = nsegs > 0 ? nsegs : 1;
    const TableView t = table_view(d_table, S);
    const int64_t ncap = build->nrows;
    const int64_t nslots = 2 * ncap + 2 * S;
    const int threads = 256;
    const unsigned init_blocks = static_cast<unsigned>(std::min<int64_t>(cdiv(nslots, threads), 8192));
    build_init_kernel<<<init_blocks, threads, 0, st>>>(t, S, unique ? 1 : 0, d_seg, build->d_nrows, ncap);
    note_launch();
    if ((s = check_launch("px_join_build init")) != PX_OK) return s;
    if (ncap > 0) {
        build_insert_kernel<<<static_cast<unsigned>(cdiv(ncap, threads)), threads, 0, st>>>(
            t, S, unique ? 1 : 0, static_cast<const int64_t*>(build->cols[pk_col].data), build->d_nrows, ncap,
            &static_cast<WsHeader*>(d_ws)->status);
        note_launch();
        if ((s = check_launch("px_join_build insert")) != PX_OK) return s;
    }
    return PX_OK;
}

px_status px_join_probe(const void* d_table, const px_batch* probe, int32_t fk_col, const int32_t* d_sel,
                        const int64_t* d_nsel, const int64_t* d_seg, int32_t nsegs, const int32_t* carry,
                        int32_t ncarry, const px_batch* build_payload, const px_batch* out, int32_t* d_probe_row,
                        int32_t* d_build_row, int64_t* d_nout, int64_t* d_out_seg, void* d_ws, size_t ws_bytes,
                        void* stream) {
    set_error("");
    px_status s = check_batch(probe, "px_join_probe probe");
    if (s != PX_OK) return s;
    if (!d_table || !aligned16(d_table)) return fail(PX_ERR_INVALID, "px_join_probe: null or misaligned table");
    if (fk_col < 0 || fk_col >= probe->ncols) return fail(PX_ERR_INVALID, "px_join_probe: fk_col %d", fk_col);
    if (probe->cols[fk_col].type != PX_I64) return fail(PX_ERR_INVALID, "px_join_probe: key column must be PX_I64");
    if ((d_sel == nullptr) != (d_nsel == nullptr))
        return fail(PX_ERR_INVALID, "px_join_probe: d_sel and d_nsel must be given together");
    if (nsegs < 0 || nsegs > PX_MAX_SEGS)
        return fail(PX_ERR_UNSUPPORTED, "px_join_probe: nsegs %d outside [0, %d]", nsegs, PX_MAX_SEGS);
    if ((nsegs > 0) != (d_seg != nullptr))
        return fail(PX_ERR_INVALID, "px_join_probe: d_seg must be given exactly when nsegs > 0");
    if (ncarry < 0 || ncarry > PX_MAX_COLS || (ncarry > 0 && !carry))
        return fail(PX_ERR_INVALID, "px_join_probe: bad carry list");
    if (build_payload && (s = check_batch(build_payload, "px_join_probe build_payload")) != PX_OK) return s;
    s = check_batch(out, "px_join_probe out");
    if (s != PX_OK) return s;
    const int npay = build_payload ? build_payload->ncols : 0;
    if (out->ncols != ncarry + npay)
        return fail(PX_ERR_INVALID, "px_join_probe: out has %d columns, %d expected", out->ncols, ncarry + npay);
    if (!d_nout) return fail(PX_ERR_INVALID, "px_join_probe: null d_nout");
    OutCols oc;
    oc.ncarry = ncarry;
    oc.npay = npay;
    for (int c = 0; c < ncarry; ++c) {
        if (carry[c] < 0 || carry[c] >= probe->ncols)
            return fail(PX_ERR_INVALID, "px_join_probe: carry[%d] = %d out of range", c, carry[c]);
        const px_col& pc = probe->cols[carry[c]];
        if (out->cols[c].type != pc.type)
            return fail(PX_ERR_INVALID, "px_join_probe: out column %d type differs from probe column %d", c, carry[c]);
        oc.carry_w[c] = pc.type;
        oc.carry_in[c] = pc.data;
        oc.carry_out[c] = out->cols[c].data;
    }
    for (int c = 0; c < npay; ++c) {
        const px_col& bc = build_payload->cols[c];
        if (out->cols[ncarry + c].type != bc.type)
            return fail(PX_ERR_INVALID, "px_join_probe: out column %d type differs from payload column %d",
                        ncarry + c, c);
        oc.pay_w[c] = bc.type;
        oc.pay_in[c] = bc.data;
        oc.pay_out[c] = out->cols[ncarry + c].data;
    }
    const int64_t ncap = probe->nrows;
    s = check_ws(d_ws, ws_bytes, px_join_probe_ws_bytes(ncap), "px_join_probe");
    if (s != PX_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int32_t S = nsegs > 0 ? nsegs : 1;
    const TableView t = table_view(const_cast<void*>(d_table), S);
    const int64_t* d_n = d_sel ? d_nsel : probe->d_nrows;
    if (ncap == 0) {
        cudaMemsetAsync(d_nout, 0, sizeof(int64_t), st);
        if (d_out_seg) cudaMemsetAsync(d_out_seg, 0, sizeof(int64_t) * (S + 1), st);
        return check_launch("px_join_probe");
    }
    const int64_t ntiles = cdiv(ncap, kTile);
    char* scratch = static_cast<char*>(d_ws) + kWsScratch;
    cudaMemsetAsync(scratch, 0, scan_scratch_bytes(ntiles), st);
    probe_kernel<<<static_cast<unsigned>(ntiles), kThreads, 0, st>>>(
        t, S, static_cast<const int64_t*>(probe->cols[fk_col].data), d_sel, d_n, ncap, d_seg, oc, d_probe_row,
        d_build_row, out->nrows, d_nout, d_out_seg, scan_scratch(scratch), &static_cast<WsHeader*>(d_ws)->status,
        ntiles, build_payload ? build_payload->nrows : 0);
    note_launch();
    if ((s = check_launch("px_join_probe")) != PX_OK) return s;
    if (d_out_seg) {
        probe_seg_tail_kernel<<<1, 256, 0, st>>>(d_seg, S, nsegs > 0 ? 1 : 0, d_n, ncap, d_nout, d_out_seg);
        note_launch();
        if ((s = check_launch("px_join_probe segments")) != PX_OK) return s;
    }
    return PX_OK;
}

}  // extern "C"
