// px_join_build / px_join_probe: the join build and probe pipelines (Sec. 3.1;
// the join-heavy queries Q5/Q9 of Sec. 3.4), per partition after the exchange
// when segments are given.
//
// Table: caller memory with the private layout of px_table.cuh (32-byte buckets
// of 2 slots: keys, build rows, payload values; segment q owns n_q + 1 buckets, so
// every segment runs at load factor < 1/2 and the whole table is n + nsegs buckets
// with no size known before the build). Linear probing over slots starts at the
// first slot of the key's home bucket: the multiply-shift reduction of the LOWER
// 32 bits of fmix64(key) (the exchange uses the upper 32) onto the segment's
// buckets. A lookup reads its home bucket's whole sector (keys, rows and payload
// values); empty slots hold the key INT64_MIN.
#include <algorithm>

#include "px_common.cuh"
#include "px_table.cuh"

namespace px {
namespace {

// ------------------------------------------------------------------ build ----

__global__ void build_init_kernel(TableView t, int32_t S, int32_t unique, const int64_t* __restrict__ d_seg,
                                  const int64_t* __restrict__ d_n, int64_t ncap, const void* pay, int32_t pay_w) {
    allow_dependents();  // the insert may launch; it waits for this grid before touching the table
    const int64_t n = actual_rows(d_n, ncap);
    const int64_t gtid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    if (gtid == 0) {
        t.hdr->magic = kMagic;
        t.hdr->nsegs = S;
        t.hdr->unique = unique;
        t.hdr->nbuild = n;
        t.hdr->pay_src = pay;
        t.hdr->pay_w = pay ? pay_w : 0;
        // Segment offsets clamped to be non-decreasing within [0, n] and to end at
        // n, so no segment can address a bucket outside the table.
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
    // Every bucket cleared whole with one 32-byte store (keys empty, rows and payload
    // values zero): whole sectors written (clearing the keys alone, 16 bytes per
    // sector, measured 10 us slower at 2M build rows).
    const int64_t nbk = table_buckets(n, S);
    longlong4_32a e;
    e.x = kEmpty;
    e.y = kEmpty;
    e.z = 0;
    e.w = 0;
    for (int64_t w = gtid; w < nbk; w += stride) *reinterpret_cast<longlong4_32a*>(&t.bk[w]) = e;
}

__global__ void build_insert_kernel(TableView t, int32_t S, int32_t unique, const int64_t* __restrict__ pk,
                                    const int64_t* __restrict__ d_n, int64_t ncap, const void* __restrict__ pay,
                                    int32_t pay_w, int32_t* status) {
    const int64_t n = actual_rows(d_n, ncap);
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t key = pk[i];  // an input of earlier calls: loaded while the clearing finishes
    wait_prior();               // the cleared buckets and the table's segment offsets
    if (key == kEmpty) {
        set_status(status, PX_ERR_UNSUPPORTED);
        return;
    }
    const int q = S > 1 ? seg_of(t.seg, S, i) : 0;
    const SegGeom g = seg_geom(t, q);
    Bucket* bk = t.bk + g.b0;
    const uint64_t nslots = uint64_t(kSlots) * g.nb;
    uint64_t s = uint64_t(kSlots) * home_bucket(static_cast<uint64_t>(key), g.nb);
    for (uint64_t probe = 0; probe < nslots; ++probe) {
        Bucket& b = bk[s / kSlots];
        const unsigned long long prev = atomicCAS(reinterpret_cast<unsigned long long*>(&b.key[s % kSlots]),
                                                  static_cast<unsigned long long>(kEmpty),
                                                  static_cast<unsigned long long>(key));
        if (prev == static_cast<unsigned long long>(kEmpty)) {
            b.row[s % kSlots] = static_cast<int32_t>(i);
            if (pay) b.pay[s % kSlots] = static_cast<int32_t>(load_int(pay, pay_w, i));
            return;
        }
        if (unique && prev == static_cast<unsigned long long>(key)) {
            set_status(status, PX_ERR_DUPLICATE_KEY);
            return;
        }
        if (++s == nslots) s = 0;
    }
    set_status(status, PX_ERR_TABLE_FULL);
}

// ------------------------------------------------------------------ probe ----
//
// Three streaming launches (plus one for the segments' first output rows), none
// of which waits on another block:
//   match - per position, find the key's build row in its segment's table and
//           record it (mrow: build row, -1 for no match, or -(slot + 2) for the
//           first of several matches in a multi-map); per-tile match counts.
//   scan  - exclusive scan of the tile counts: each tile's first output row.
//   emit  - per tile, a block scan of the per-position match counts gives every
//           output row; carried probe columns and gathered payload columns are
//           written column by column, every load of a column before its stores.
// The extra 4 bytes written and read per position buy the removal of the
// serialised look-back that stalled a single-pass probe: a block of a single
// pass alternates latency-bound lookups and DRAM-bound emission behind its
// barriers, while separate kernels each run at full occupancy.

constexpr int kThreads = 256;
constexpr int kItems = 4;
constexpr int kTile = kThreads * kItems;  // 1024 positions
constexpr int kWarps = kThreads / 32;
constexpr int32_t kNoMatch = -1;

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

template <typename T>
__device__ __forceinline__ void gather_store_t(const void* in, void* out, const int32_t* src, const int64_t* dst,
                                               const bool* ok) {
    T v[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i)
        if (ok[i]) v[i] = static_cast<const T*>(in)[src[i]];
#pragma unroll
    for (int i = 0; i < kItems; ++i)
        if (ok[i]) static_cast<T*>(out)[dst[i]] = v[i];
}

// out[dst[i]] = in[src[i]] for the items with ok[i], all loads before the stores.
__device__ __forceinline__ void gather_store(int w, const void* in, void* out, const int32_t* src, const int64_t* dst,
                                             const bool* ok) {
    if (w == 8) gather_store_t<int64_t>(in, out, src, dst, ok);
    else if (w == 4) gather_store_t<int32_t>(in, out, src, dst, ok);
    else gather_store_t<int8_t>(in, out, src, dst, ok);
}

__device__ __forceinline__ void emit(const OutCols& oc, int64_t pos, int64_t prow, int64_t brow,
                                     int32_t* probe_row, int32_t* build_row) {
    if (probe_row) probe_row[pos] = static_cast<int32_t>(prow);
    if (build_row) build_row[pos] = static_cast<int32_t>(brow);
    for (int c = 0; c < oc.ncarry; ++c) copy_cell(oc.carry_out[c], oc.carry_in[c], oc.carry_w[c], pos, prow);
    for (int c = 0; c < oc.npay; ++c) copy_cell(oc.pay_out[c], oc.pay_in[c], oc.pay_w[c], pos, brow);
}

// Number of matches of `key` along the probe sequence from slot `s` (numbered
// within the segment's buckets), and the slot of the first one. Multi-map tables
// hold fewer than 2^30 rows, so segment slot numbers fit 32 bits.
__device__ __forceinline__ int32_t count_matches(const Bucket* segb, uint32_t nb, uint32_t s, int64_t key,
                                                 uint32_t* first) {
    const uint32_t nslots = kSlots * nb;
    int32_t m = 0;
    for (uint32_t probe = 0; probe < nslots; ++probe) {
        const int64_t k = segb[s / kSlots].key[s % kSlots];
        if (k == key) {
            if (m == 0) *first = s;
            ++m;
        } else if (k == kEmpty) {
            break;
        }
        if (++s == nslots) s = 0;
    }
    return m;
}

constexpr int kMatchThreads = 512;
constexpr int kMatchItems = kTile / kMatchThreads;  // positions per thread per tile (same tiles as emit)

// Keys of this thread's positions of the tile whose first position is j0 (kEmpty
// where there is no row).
template <bool kSel>
__device__ __forceinline__ void match_keys(const int64_t* __restrict__ fk, const int32_t* __restrict__ sel,
                                           uint32_t n, uint32_t j0, int64_t* keyv) {
#pragma unroll
    for (int i = 0; i < kMatchItems; ++i) {
        const uint32_t j = j0 + 32 * i;
        keyv[i] = j < n ? fk[kSel ? static_cast<uint32_t>(sel[j]) : j] : kEmpty;
    }
}

// Segment cursor of one thread: segment q holds the thread's latest position,
// `end` is where q's positions end, segb/nb are q's buckets. A thread's positions
// only increase, so the cursor only moves forward.
struct SegCursor {
    int q;
    int64_t end;
    const Bucket* segb;
    uint32_t nb;
};

__device__ __forceinline__ void cursor_geom(SegCursor& c, const TableView& t) {
    const SegGeom g = seg_geom(t, c.q);
    c.segb = t.bk + g.b0;
    c.nb = g.nb;
}

__device__ __forceinline__ void cursor_init(SegCursor& c, const TableView& t, const int64_t* pseg, int S, int64_t j) {
    c.q = S > 1 ? seg_of(pseg, S, j) : 0;
    c.end = c.q + 1 < S ? pseg[c.q + 1] : INT64_MAX;
    cursor_geom(c, t);
}

__device__ __forceinline__ void cursor_seek(SegCursor& c, const TableView& t, const int64_t* pseg, int S, int64_t j) {
    if (j < c.end) return;
    do {
        ++c.q;
        c.end = c.q + 1 < S ? pseg[c.q + 1] : INT64_MAX;
    } while (j >= c.end);
    cursor_geom(c, t);
}

// Walks on from home bucket `hb` of a segment (a bucket full without the key)
// through the following buckets: the key's build row, or kNoMatch at the first
// empty slot. Occupied slots form a prefix of every probe sequence.
__device__ __forceinline__ int32_t walk_on(const Bucket* segb, uint32_t nb, uint32_t hb, int64_t key) {
    BucketRegs v;
    const int l = walk_find(segb, nb, hb, key, &v);
    return l >= 0 ? bucket_row(v, l) : kNoMatch;
}

// Persistent over tiles (grid-stride), software-pipelined: the next tile's keys
// are loaded while the current tile's buckets are in flight. No block-wide
// barrier: every thread reads the (cached) table header once and follows its own
// segment cursor (one check per tile when all of the thread's positions lie in
// its current segment); warps add their match counts atomically. Unique tables:
// every position reads its home bucket's keys and rows (two sectors, one round
// trip); the few keys whose home bucket is full without them walk on inline,
// only in warps where some lane needs it. Only positions below the row count are
// written: the emit reads no other.
template <bool kSel>
__global__ void __launch_bounds__(kMatchThreads, 3)
probe_match_kernel(TableView t, int32_t S, const int64_t* __restrict__ fk, const int32_t* __restrict__ sel,
                   const int64_t* __restrict__ d_n, int64_t ncap, const int64_t* __restrict__ pseg,
                   int32_t* __restrict__ mrow, int32_t* __restrict__ tile_cnt, int32_t* status, int32_t npay,
                   int64_t payload_rows, uint32_t ntiles) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n = actual_rows(d_n, ncap);
    const bool bad = t.hdr->magic != kMagic || t.hdr->nsegs != S || (npay > 0 && t.hdr->nbuild > payload_rows);
    if (bad && blockIdx.x == 0 && threadIdx.x == 0) set_status(status, PX_ERR_INVALID);
    const bool unique = t.hdr->unique != 0;
    // Positions fit 32 bits (batches hold at most INT32_MAX rows); item i of a tile
    // sits at tile * kTile + lane_off + 32 i.
    const uint32_t lane_off = warp * (32 * kMatchItems) + lane;
    const uint32_t nv = static_cast<uint32_t>(n);  // positions with a key to look up
    uint32_t tile = blockIdx.x;
    if (bad) {  // a table this call cannot use: no matches, and no reads past its header
        for (; tile < ntiles; tile += gridDim.x)
#pragma unroll
            for (int i = 0; i < kMatchItems; ++i) {
                const uint32_t j = tile * kTile + lane_off + 32 * i;
                if (j < nv) mrow[j] = kNoMatch;
            }
        return;
    }
    if (tile >= ntiles) return;
    SegCursor c;
    cursor_init(c, t, pseg, S, tile * kTile + lane_off);
    int64_t keyv[kMatchItems];
    match_keys<kSel>(fk, sel, nv, tile * kTile + lane_off, keyv);
    for (; tile < ntiles; tile += gridDim.x) {
        const uint32_t j0 = tile * kTile + lane_off;
        const Bucket* segb[kMatchItems];
        uint32_t nb[kMatchItems];
        if (static_cast<int64_t>(j0 + 32 * (kMatchItems - 1)) < c.end) {
#pragma unroll
            for (int i = 0; i < kMatchItems; ++i) {
                segb[i] = c.segb;
                nb[i] = c.nb;
            }
        } else {
#pragma unroll
            for (int i = 0; i < kMatchItems; ++i) {
                cursor_seek(c, t, pseg, S, j0 + 32 * i);
                segb[i] = c.segb;
                nb[i] = c.nb;
            }
        }
        uint32_t hb[kMatchItems];  // home bucket, numbered within the segment
#pragma unroll
        for (int i = 0; i < kMatchItems; ++i) hb[i] = home_bucket(static_cast<uint64_t>(keyv[i]), nb[i]);
        int32_t out[kMatchItems];
        int32_t cnt = 0;
        if (unique) {
            // Every home bucket is read whole (one sector: keys and rows); hb < nb
            // keeps the reads inside the segment even for positions without a key.
            BucketRegs bv[kMatchItems];
#pragma unroll
            for (int i = 0; i < kMatchItems; ++i) bv[i] = load_bucket(segb[i] + hb[i]);
            // Next tile's keys go out while this tile's buckets are in flight.
            int64_t keyn[kMatchItems];
            match_keys<kSel>(fk, sel, nv, (tile + gridDim.x) * kTile + lane_off, keyn);
            uint32_t pend = 0;  // items whose home bucket is full without their key
#pragma unroll
            for (int i = 0; i < kMatchItems; ++i) {
                const bool live = keyv[i] != kEmpty;  // a row, and not the reserved key
                // a unique table holds a key at most once: the compares select unordered
                int32_t r = bv[i].k0 == keyv[i] ? bv[i].r0 : kNoMatch;
                r = bv[i].k1 == keyv[i] ? bv[i].r1 : r;
                out[i] = live ? r : kNoMatch;
                if (live && r < 0 && bv[i].k1 != kEmpty) pend |= 1u << i;
            }
            if (__any_sync(FULL, pend != 0)) {
#pragma unroll
                for (int i = 0; i < kMatchItems; ++i)
                    if ((pend >> i) & 1u) out[i] = walk_on(segb[i], nb[i], hb[i], keyv[i]);
            }
#pragma unroll
            for (int i = 0; i < kMatchItems; ++i) {
                cnt += out[i] >= 0 ? 1 : 0;
                keyv[i] = keyn[i];
            }
        } else {
            // Multi-map: count every match; one match is recorded as its build row,
            // several as -(table slot of the first + 2) for the emit pass to walk.
#pragma unroll
            for (int i = 0; i < kMatchItems; ++i) {
                out[i] = kNoMatch;
                if (keyv[i] == kEmpty) continue;
                uint32_t first = 0;
                const int32_t m = count_matches(segb[i], nb[i], kSlots * hb[i], keyv[i], &first);
                const int64_t b0 = segb[i] - t.bk;
                if (m == 1) out[i] = segb[i][first / kSlots].row[first % kSlots];
                else if (m > 1) out[i] = -static_cast<int32_t>(kSlots * b0 + first) - 2;
                cnt += m;
            }
            match_keys<kSel>(fk, sel, nv, (tile + gridDim.x) * kTile + lane_off, keyv);
        }
        cnt = static_cast<int32_t>(__reduce_add_sync(FULL, static_cast<uint32_t>(cnt)));
        if (lane == 0 && cnt) atomicAdd(&tile_cnt[tile], cnt);  // zeroed before the launch
#pragma unroll
        for (int i = 0; i < kMatchItems; ++i) {
            const uint32_t j = j0 + 32 * i;
            if (j < nv) mrow[j] = out[i];
        }
    }
}

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan of the tile counts (single pass, bounded look-back); the last
// tile writes the total to *d_nout and flags an output over capacity.
__global__ void __launch_bounds__(kScanThreads)
probe_scan_kernel(const int32_t* __restrict__ cnt, int64_t* __restrict__ off, int64_t total, int64_t out_cap,
                  int64_t* __restrict__ d_nout, ScanScratch scan, int32_t* status, int64_t nscan_tiles) {
    __shared__ int64_t s_tile;
    __shared__ int64_t s_warp[kScanThreads / 32];
    __shared__ int64_t s_excl;
    wait_prior();        // the match kernel's tile counts
    allow_dependents();  // the emit may launch and start its own loads
    const int64_t tile = next_tile(scan.counter, &s_tile);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = tile * kScanTile + static_cast<int64_t>(tid) * kScanItems;
    int64_t v[kScanItems];
    int64_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < total ? cnt[base + k] : 0;
        sum += v[k];
    }
    const int64_t incl = warp_incl_scan(sum);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int64_t w = lane < kScanThreads / 32 ? s_warp[lane] : 0;
        const int64_t wi = warp_incl_scan(w);
        if (lane < kScanThreads / 32) s_warp[lane] = wi - w;
        const int64_t agg = __shfl_sync(FULL, wi, 31);
        const int64_t excl = lookback(scan.states, tile, agg, status);
        if (lane == 0) {
            s_excl = excl;
            if (tile == nscan_tiles - 1) {
                *d_nout = excl + agg;
                if (excl + agg > out_cap) set_status(status, PX_ERR_CAPACITY);
            }
        }
    }
    __syncthreads();
    int64_t run = s_excl + s_warp[warp] + incl - sum;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < total) off[base + k] = run;
        run += v[k];
    }
}
// Output rows of one tile in position order. A tile whose every position matched
// exactly once in a unique table (its count equals its rows) writes output row
// tile_off + position - tile start, with no ranking. Other tiles rank their
// matches: unique matches count 0 or 1, so a ballot per item ranks them; a warp
// holding a multi-map position (several matches, counted again along its chain)
// takes shuffle scans instead.
template <bool kSel>
__global__ void __launch_bounds__(kThreads)
probe_emit_kernel(TableView t, int32_t S, const int64_t* __restrict__ fk, const int32_t* __restrict__ sel,
                  const int64_t* __restrict__ d_n, int64_t ncap, const int64_t* __restrict__ pseg,
                  const int32_t* __restrict__ mrow, const int32_t* __restrict__ tile_cnt,
                  const int64_t* __restrict__ tile_off, OutCols oc, int32_t* __restrict__ probe_row,
                  int32_t* __restrict__ build_row, int64_t out_cap) {
    __shared__ int32_t s_warp[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n = actual_rows(d_n, ncap);
    // Positions fit 32 bits (batches hold at most INT32_MAX rows).
    const uint32_t tb = static_cast<uint32_t>(blockIdx.x) * kTile;
    const int rows = n - tb >= kTile ? kTile : static_cast<int>(n - tb);  // valid positions in this tile (<= 0: none)
    if (rows <= 0) return;
    int lp[kItems];  // position within the tile
    int32_t mr[kItems], prow[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        lp[i] = warp * (32 * kItems) + i * 32 + lane;
        prow[i] = lp[i] < rows ? (kSel ? sel[tb + lp[i]] : static_cast<int32_t>(tb + lp[i])) : 0;
    }
    // The join's common shape (one 8-byte carried column, one 4-byte payload column):
    // every position's carried value is loaded first (an input of earlier calls, so
    // before the wait for the scan: it overlaps the scan's tail), then the match rows
    // and the payload gathers, whose latency overlaps the ranking and block combine.
    const bool early = oc.ncarry == 1 && oc.npay == 1 && oc.carry_w[0] == 8 && oc.pay_w[0] == 4;
    int64_t cv[kItems];
    int32_t pv[kItems];
    if (early) {
#pragma unroll
        for (int i = 0; i < kItems; ++i)
            if (lp[i] < rows) cv[i] = static_cast<const int64_t*>(oc.carry_in[0])[prow[i]];
    }
    wait_prior();  // the scan's tile offsets, and the match rows and counts before them
    allow_dependents();
#pragma unroll
    for (int i = 0; i < kItems; ++i) mr[i] = lp[i] < rows ? mrow[tb + lp[i]] : kNoMatch;
    if (early) {
#pragma unroll
        for (int i = 0; i < kItems; ++i)
            if (mr[i] >= 0) pv[i] = static_cast<const int32_t*>(oc.pay_in[0])[mr[i]];
    }
    const int64_t tile_base = tile_off[blockIdx.x];
    int64_t pos[kItems];
    bool one[kItems];
    int32_t m[kItems];
    int64_t key[kItems];
    bool multi = false;
    if (tile_cnt[blockIdx.x] == rows && t.hdr->unique != 0) {
        // Every position of the tile matched once: no ranking, no block combine.
        const int64_t room = out_cap - tile_base;  // output rows left from this tile's first
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            pos[i] = tile_base + lp[i];
            one[i] = lp[i] < rows && lp[i] < room;
        }
    } else {
        bool has_multi = false;
#pragma unroll
        for (int i = 0; i < kItems; ++i) has_multi |= mr[i] < kNoMatch;
        multi = __any_sync(FULL, has_multi);
        int32_t pre[kItems];
        int32_t wsum = 0;
        if (!multi) {
            const uint32_t lt = lanemask_lt();
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                m[i] = mr[i] >= 0 ? 1 : 0;
                const uint32_t b = __ballot_sync(FULL, m[i] != 0);
                pre[i] = wsum + __popc(b & lt);
                wsum += __popc(b);
            }
        } else {
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                m[i] = mr[i] >= 0 ? 1 : 0;
                key[i] = 0;
                if (mr[i] < kNoMatch) {
                    const SegGeom g = seg_geom(t, S > 1 ? seg_of(pseg, S, tb + lp[i]) : 0);
                    const uint32_t first = static_cast<uint32_t>(-static_cast<int64_t>(mr[i]) - 2 - kSlots * g.b0);
                    key[i] = fk[prow[i]];
                    uint32_t dummy = 0;
                    m[i] = count_matches(t.bk + g.b0, g.nb, first, key[i], &dummy);
                }
                const int32_t incl = warp_incl_scan(m[i]);
                pre[i] = wsum + incl - m[i];
                wsum += __shfl_sync(FULL, incl, 31);
            }
        }
        // Block combine; the tile's first row comes from the scan of the tile counts.
        if (lane == 0) s_warp[warp] = wsum;
        __syncthreads();
        int32_t wb = lane < warp ? s_warp[lane] : 0;  // totals of the warps before this one, in lanes < kWarps
#pragma unroll
        for (int d = 1; d < kWarps; d <<= 1) wb += __shfl_xor_sync(FULL, wb, d);
        wb = __shfl_sync(FULL, wb, 0);
        const int64_t base = tile_base + wb;
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            pos[i] = base + pre[i];
            one[i] = mr[i] >= 0 && pos[i] < out_cap;
        }
    }
    if (probe_row) {
#pragma unroll
        for (int i = 0; i < kItems; ++i)
            if (one[i]) probe_row[pos[i]] = prow[i];
    }
    if (build_row) {
#pragma unroll
        for (int i = 0; i < kItems; ++i)
            if (one[i]) build_row[pos[i]] = mr[i];
    }
    if (early) {
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            if (one[i]) {
                static_cast<int64_t*>(oc.carry_out[0])[pos[i]] = cv[i];
                static_cast<int32_t*>(oc.pay_out[0])[pos[i]] = pv[i];
            }
        }
    } else {
        for (int c = 0; c < oc.ncarry; ++c)
            gather_store(oc.carry_w[c], oc.carry_in[c], oc.carry_out[c], prow, pos, one);
        for (int c = 0; c < oc.npay; ++c) gather_store(oc.pay_w[c], oc.pay_in[c], oc.pay_out[c], mr, pos, one);
    }
    if (!multi) return;
    // Positions with several matches: walk the chain again, emitting each.
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        if (mr[i] >= kNoMatch) continue;
        const SegGeom g = seg_geom(t, S > 1 ? seg_of(pseg, S, tb + lp[i]) : 0);
        const Bucket* segb = t.bk + g.b0;
        const uint32_t nslots = kSlots * g.nb;
        uint32_t s = static_cast<uint32_t>(-static_cast<int64_t>(mr[i]) - 2 - kSlots * g.b0);
        int64_t p = pos[i];
        for (uint32_t probe = 0; probe < nslots && p < pos[i] + m[i]; ++probe) {
            const int64_t k = segb[s / kSlots].key[s % kSlots];
            if (k == key[i]) {
                if (p < out_cap) emit(oc, p, prow[i], segb[s / kSlots].row[s % kSlots], probe_row, build_row);
                ++p;
            } else if (k == kEmpty) {
                break;
            }
            if (++s == nslots) s = 0;
        }
    }
}

// First output row of every segment (out_seg[q], q in [0, S]): the output rows of
// the positions before the segment's first position, i.e. its tile's first output
// row plus the matches of the tile's positions before it; nout for a segment that
// starts at or past the last position. One block per segment, one thread per
// position of the tile.
__global__ void __launch_bounds__(kTile)
probe_seg_kernel(TableView t, int32_t S, int32_t segmented, const int64_t* __restrict__ pseg,
                 const int64_t* __restrict__ fk, const int32_t* __restrict__ sel, const int64_t* __restrict__ d_n,
                 int64_t ncap, const int32_t* __restrict__ mrow, const int64_t* __restrict__ tile_off,
                 const int64_t* __restrict__ d_nout, int64_t* __restrict__ d_out_seg) {
    __shared__ int32_t s_warp[kTile / 32];
    wait_prior();  // the match rows, tile offsets and row count
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q = blockIdx.x;
    const int64_t n = actual_rows(d_n, ncap);
    int64_t start = segmented ? pseg[q] : (q == 0 ? 0 : n);
    start = start < 0 ? 0 : start;
    if (start >= n) {
        if (threadIdx.x == 0) d_out_seg[q] = *d_nout;
        return;
    }
    const int64_t j = start / kTile * kTile + threadIdx.x;
    int32_t cnt = 0;
    if (j < start) {
        const int32_t r = mrow[j];
        if (r >= 0) {
            cnt = 1;
        } else if (r < kNoMatch) {  // first of several matches: count them along the chain
            const SegGeom g = seg_geom(t, S > 1 ? seg_of(pseg, S, j) : 0);
            const uint32_t first = static_cast<uint32_t>(-static_cast<int64_t>(r) - 2 - kSlots * g.b0);
            uint32_t dummy = 0;
            cnt = count_matches(t.bk + g.b0, g.nb, first, fk[sel ? static_cast<int64_t>(sel[j]) : j], &dummy);
        }
    }
    cnt = static_cast<int32_t>(__reduce_add_sync(FULL, static_cast<uint32_t>(cnt)));
    if (lane == 0) s_warp[warp] = cnt;
    __syncthreads();
    if (warp == 0) {
        cnt = static_cast<int32_t>(__reduce_add_sync(FULL, static_cast<uint32_t>(s_warp[lane])));
        if (lane == 0) d_out_seg[q] = tile_off[start / kTile] + cnt;
    }
}

// Probe workspace: [header][mrow: 4 B per position][tile counts][tile offsets]
// [scan scratch over the tile counts].
struct ProbeWs {
    size_t mrow, cnt, off, scan, total;
    int64_t ntiles, nscan;
};

ProbeWs probe_ws_layout(int64_t nprobe) {
    if (nprobe < 0) nprobe = 0;
    ProbeWs L;
    L.ntiles = cdiv(nprobe, kTile);
    L.nscan = cdiv(L.ntiles, kScanTile);
    L.mrow = kWsScratch;
    L.cnt = L.mrow + align_up(4 * static_cast<size_t>(nprobe), 256);
    L.off = L.cnt + align_up(4 * static_cast<size_t>(L.ntiles), 256);
    L.scan = L.off + align_up(8 * static_cast<size_t>(L.ntiles), 256);
    L.total = L.scan + scan_scratch_bytes(L.nscan);
    return L;
}

}  // namespace
}  // namespace px

using namespace px;

extern "C" {

size_t px_join_table_bytes(int64_t nbuild, int32_t nsegs) {
    if (nbuild < 0) nbuild = 0;
    const int32_t S = nsegs > 0 ? nsegs : 1;
    return 64 + seg_area_bytes(S) + 16 + static_cast<size_t>(table_buckets(nbuild, S)) * sizeof(Bucket);
}

size_t px_join_build_ws_bytes(int64_t nbuild) {
    (void)nbuild;
    return kWsScratch;
}

size_t px_join_probe_ws_bytes(int64_t nprobe) {
    return probe_ws_layout(nprobe).total;
}

px_status px_join_build(const px_batch* build, int32_t pk_col, const int64_t* d_seg, int32_t nsegs, int32_t unique,
                        int32_t pay_col, void* d_table, size_t table_bytes, void* d_ws, size_t ws_bytes,
                        void* stream) {
    CallRange nvtx_range("px_join_build");
    set_error("");
    px_status s = check_batch(build, "px_join_build build");
    if (s != PX_OK) return s;
    if (pk_col < 0 || pk_col >= build->ncols) return fail(PX_ERR_INVALID, "px_join_build: pk_col %d", pk_col);
    if (build->cols[pk_col].type != PX_I64) return fail(PX_ERR_INVALID, "px_join_build: key column must be PX_I64");
    if (pay_col < -1 || pay_col >= build->ncols || pay_col == pk_col)
        return fail(PX_ERR_INVALID, "px_join_build: pay_col %d", pay_col);
    if (pay_col >= 0 && build->cols[pay_col].type != PX_I8 && build->cols[pay_col].type != PX_I32)
        return fail(PX_ERR_UNSUPPORTED, "px_join_build: the copied payload column must be PX_I8 or PX_I32");
    const void* pay = pay_col >= 0 ? build->cols[pay_col].data : nullptr;
    const int32_t pay_w = pay_col >= 0 ? build->cols[pay_col].type : 0;
    if (nsegs < 0 || nsegs > PX_MAX_SEGS)
        return fail(PX_ERR_UNSUPPORTED, "px_join_build: nsegs %d outside [0, %d]", nsegs, PX_MAX_SEGS);
    if ((nsegs > 0) != (d_seg != nullptr))
        return fail(PX_ERR_INVALID, "px_join_build: d_seg must be given exactly when nsegs > 0");
    if (!d_table || !aligned16(d_table)) return fail(PX_ERR_INVALID, "px_join_build: null or misaligned table");
    if (table_bytes < px_join_table_bytes(build->nrows, nsegs))
        return fail(PX_ERR_INVALID, "px_join_build: table of %zu bytes, %zu needed", table_bytes,
                    px_join_table_bytes(build->nrows, nsegs));
    if (!unique && kSlots * table_buckets(build->nrows, nsegs > 0 ? nsegs : 1) + 2 > INT32_MAX)
        return fail(PX_ERR_UNSUPPORTED, "px_join_build: multi-map tables hold below about 2^30 rows");
    s = check_ws(d_ws, ws_bytes, px_join_build_ws_bytes(build->nrows), "px_join_build");
    if (s != PX_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int32_t S = nsegs > 0 ? nsegs : 1;
    const TableView t = table_view(d_table, S);
    const int64_t ncap = build->nrows;
    const int64_t nwords = table_buckets(ncap, S);  // buckets whose keys to clear
    const int threads = 256;
    const unsigned init_blocks = static_cast<unsigned>(std::min<int64_t>(cdiv(nwords, threads), 8192));
    build_init_kernel<<<init_blocks, threads, 0, st>>>(t, S, unique ? 1 : 0, d_seg, build->d_nrows, ncap, pay, pay_w);
    note_launch();
    if ((s = check_launch("px_join_build init")) != PX_OK) return s;
    if (ncap > 0) {
        launch_after(build_insert_kernel, dim3(static_cast<unsigned>(cdiv(ncap, threads))), dim3(threads), 0, st, t, S,
                     unique ? 1 : 0, static_cast<const int64_t*>(build->cols[pk_col].data), build->d_nrows, ncap,
                     pay, pay_w, &static_cast<WsHeader*>(d_ws)->status);
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
    CallRange nvtx_range("px_join_probe");
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
    const ProbeWs L = probe_ws_layout(ncap);
    char* ws = static_cast<char*>(d_ws);
    int32_t* mrow = reinterpret_cast<int32_t*>(ws + L.mrow);
    int32_t* tcnt = reinterpret_cast<int32_t*>(ws + L.cnt);
    int64_t* toff = reinterpret_cast<int64_t*>(ws + L.off);
    int32_t* status = &static_cast<WsHeader*>(d_ws)->status;
    const int64_t* fk = static_cast<const int64_t*>(probe->cols[fk_col].data);
    const unsigned grid = static_cast<unsigned>(L.ntiles);
    cudaMemsetAsync(tcnt, 0, 4 * static_cast<size_t>(L.ntiles), st);
    cudaMemsetAsync(ws + L.scan, 0, scan_scratch_bytes(L.nscan), st);  // before the match: the scan follows it directly
    const bool has_sel = d_sel != nullptr;
    const auto match = has_sel ? probe_match_kernel<true> : probe_match_kernel<false>;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, match, kMatchThreads, 0);
    const unsigned mgrid = static_cast<unsigned>(std::min<int64_t>(L.ntiles, int64_t(sm_count()) * std::max(1, per_sm)));
    match<<<mgrid, kMatchThreads, 0, st>>>(t, S, fk, d_sel, d_n, ncap, d_seg, mrow, tcnt, status, npay,
                                           build_payload ? build_payload->nrows : 0, static_cast<uint32_t>(L.ntiles));
    note_launch();
    if ((s = check_launch("px_join_probe match")) != PX_OK) return s;
    launch_after(probe_scan_kernel, dim3(static_cast<unsigned>(L.nscan)), dim3(kScanThreads), 0, st, tcnt, toff,
                 L.ntiles, out->nrows, d_nout, scan_scratch(ws + L.scan), status, L.nscan);
    note_launch();
    if ((s = check_launch("px_join_probe scan")) != PX_OK) return s;
    const auto emit = has_sel ? probe_emit_kernel<true> : probe_emit_kernel<false>;
    launch_after(emit, dim3(grid), dim3(kThreads), 0, st, t, S, fk, d_sel, d_n, ncap, d_seg, mrow, tcnt, toff, oc,
                 d_probe_row, d_build_row, out->nrows);
    note_launch();
    if ((s = check_launch("px_join_probe emit")) != PX_OK) return s;
    if (d_out_seg) {
        launch_after(probe_seg_kernel, dim3(static_cast<unsigned>(S + 1)), dim3(kTile), 0, st, t, S, nsegs > 0 ? 1 : 0,
                     d_seg, fk, d_sel, d_n, ncap, mrow, toff, d_nout, d_out_seg);
        note_launch();
        if ((s = check_launch("px_join_probe segments")) != PX_OK) return s;
    }
    return PX_OK;
}

}  // extern "C"
