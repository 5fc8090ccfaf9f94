// px_fragments_run: a batch of independent plan fragments, each FilterProject ->
// join probe -> HashAggregation (Single mode) over one probe batch and one
// prebuilt dimension table (the operators of Sec. 3.2 and the join probe
// pipeline of Sec. 3.1), run as ONE persistent fused kernel plus one emit kernel.
// The paper finds small vectors leave a GPU underused (Sec. 3.3.2) and results
// sensitive to batch size (Sec. 3.4); batching whole fragments into one launch is
// this library's answer for many small fragments.
//
// Work items are (fragment, chunk of rows), handed out by a device counter in
// the order of decreasing fragment size. A block walks its chunk in tiles of
// THREADS x ITEMS rows: per row the filter column, join key and aggregate inputs
// load together, then the key's home bucket (one sector: keys, build rows and,
// when the dimension was built with its group column copied, the group keys),
// else the group key gathered from the build column at the build row; the
// aggregates go into the fragment's dense accumulators (group key - group_lo
// indexes them):
//   * shared mode (small key ranges): block arrays in shared memory, cleared per
//     work item and added into the fragment's global arrays at its end;
//   * direct mode: 64-bit reductions straight into the global arrays.
// Rows of one warp that share lane 0's group are summed with a butterfly first.
// The emit kernel compacts each fragment's occupied slots into its output in
// key order (single pass, per-fragment bounded look-back).
#include <algorithm>
#include <vector>

#include "px_common.cuh"
#include "px_table.cuh"

namespace px {
namespace {

constexpr size_t kSmemAccBudget = 96 * 1024;  // shared-mode block accumulators
constexpr int kEmitThreads = 256;
constexpr int kEmitItems = 8;
constexpr int kEmitTile = kEmitThreads * kEmitItems;
constexpr int kMajority = 6;  // smallest lane group worth a warp reduction

// Device plan of one fragment.
struct FragDev {
    const int64_t* key;
    const void* filter;
    int64_t lo, hi;
    int64_t nrows;
    // aggregate k reads column pa[k] (width wa[k]) and, for SUM_MUL, pb[k] (wb[k])
    const void* pa[PX_FRAG_MAX_AGGS];
    const void* pb[PX_FRAG_MAX_AGGS];
    int32_t op[PX_FRAG_MAX_AGGS], wa[PX_FRAG_MAX_AGGS], wb[PX_FRAG_MAX_AGGS];
    int32_t filter_w, naggs, group_w, count_agg;  // count_agg: a COUNT aggregate, or -1
    TableView t;
    int64_t nbuild;
    const void* group;
    int64_t group_lo;
    uint32_t D;      // dense slots
    int32_t shared;  // 1: block accumulators in shared memory
    int64_t chunk;   // rows per work item
    unsigned long long* acc;  // [naggs][D]
    uint8_t* occ;             // [D] occupancy flags (only without COUNT)
    uint64_t* emit_states;    // look-back states of the fragment's emit tiles
    void* out_keys;
    int64_t* out_aggs[PX_FRAG_MAX_AGGS];
    int64_t* ngroups;
    int64_t max_groups;
};

struct PlanHeader {
    int32_t nfrags;
    int32_t reserved;
    int64_t nitems;  // work items
    int64_t nemit;   // emit tiles
    int64_t pad[5];
};

// Plan (host staging and its device copy): header, item_start[nfrags + 1],
// emit_start[nfrags + 1], FragDev[nfrags]; fragments in work order.
struct PlanLayout {
    size_t items, emits, frags, total;
};
PlanLayout plan_layout(int32_t n) {
    PlanLayout L;
    L.items = sizeof(PlanHeader);
    L.emits = L.items + align_up(8 * static_cast<size_t>(n + 1), 64);
    L.frags = L.emits + align_up(8 * static_cast<size_t>(n + 1), 64);
    L.total = L.frags + align_up(sizeof(FragDev) * static_cast<size_t>(n), 64);
    return L;
}

// Largest p with start[p] <= x (start ascending, start[0] = 0 <= x).
__device__ __forceinline__ int find_frag(const int64_t* start, int n, int64_t x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int64_t load_w(const void* p, int w, int64_t i) { return load_int(p, w, i); }

// Adds x (mod 2^64) to a 64-bit value held as 32-bit words lo/hi in shared memory.
__device__ __forceinline__ void add_split(uint32_t* lo, uint32_t* hi, uint64_t x) {
    const uint32_t xl = static_cast<uint32_t>(x), xh = static_cast<uint32_t>(x >> 32);
    const uint32_t old = atomicAdd(lo, xl);
    const uint32_t add_hi = xh + (old + xl < old ? 1u : 0u);
    if (add_hi) red_add_shared(hi, add_hi);
}

// Build row of `key` (not kEmpty) in an unsegmented unique table, or -1; *pay
// receives the payload value copied beside the key (meaningful when the table
// holds one).
__device__ __forceinline__ int32_t probe_row(const TableView& t, uint32_t nb, int64_t key, int32_t* pay) {
    const Bucket* bp = t.bk + home_bucket(static_cast<uint64_t>(key), nb);
    for (uint32_t round = 0; round < nb; ++round) {
        const BucketRegs v = load_bucket(bp);
        bool end;
        const int l = bucket_find(v, key, &end);
        if (l >= 0) {
            *pay = bucket_pay(v, l);
            return bucket_row(v, l);
        }
        if (end) return -1;
        bp = bp + 1 == t.bk + nb ? t.bk : bp + 1;
    }
    return -1;
}

// Rows [r0, r1) of fragment f. SHARED: accumulate into the block arrays lo/hi
// ([naggs][D] each) and occupancy bits; else reduce into the global arrays.
template <int THREADS, int ITEMS, int NA, bool SHARED>
__device__ void frag_rows(const FragDev& f, int64_t r0, int64_t r1, uint32_t* s_lo, uint32_t* s_hi,
                          uint32_t* s_occ, int32_t* status) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t nb = static_cast<uint32_t>(table_buckets(f.t.hdr->nbuild, 1));
    // the group column copied into the table at build time: read with the key
    const bool group_in_table = f.t.hdr->pay_src == f.group && f.t.hdr->pay_w == f.group_w;
    const int naggs = f.naggs;
    for (int64_t tb = r0; tb < r1; tb += THREADS * ITEMS) {
        int64_t key[ITEMS], v[NA][ITEMS];
        bool pass[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const int64_t r = tb + warp * (32 * ITEMS) + i * 32 + lane;
            const bool valid = r < r1;
            bool p = valid;
            if (f.filter && valid) {
                const int64_t x = load_w(f.filter, f.filter_w, r);
                p = x >= f.lo && x < f.hi;
            }
            pass[i] = p;
            key[i] = valid ? f.key[r] : kEmpty;
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                if (a >= naggs) break;
                int64_t x = 1;
                if (f.op[a] != PX_COUNT && valid) {
                    x = load_w(f.pa[a], f.wa[a], r);
                    if (f.op[a] == PX_SUM_MUL)
                        x = static_cast<int64_t>(static_cast<uint64_t>(x) *
                                                 static_cast<uint64_t>(load_w(f.pb[a], f.wb[a], r)));
                }
                v[a][i] = x;
            }
        }
        uint32_t slot[ITEMS];  // dense slot of the row's group, or 0xffffffff
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            slot[i] = 0xffffffffu;
            if (!pass[i] || key[i] == kEmpty) continue;
            int32_t pay = 0;
            const int32_t br = probe_row(f.t, nb, key[i], &pay);
            if (br < 0) continue;
            const int64_t gk = group_in_table ? static_cast<int64_t>(pay) : load_w(f.group, f.group_w, br);
            const uint64_t d = static_cast<uint64_t>(gk - f.group_lo);
            if (d < f.D) slot[i] = static_cast<uint32_t>(d);
            else set_status(status, PX_ERR_UNSUPPORTED);
        }
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            // Rows sharing lane 0's slot: one butterfly sum, applied once by lane 0.
            uint32_t apply = slot[i];
            const uint32_t c0 = __shfl_sync(FULL, slot[i], 0);
            const uint32_t mm = __ballot_sync(FULL, slot[i] == c0);
            if (c0 != 0xffffffffu && __popc(mm) >= kMajority) {
                const bool in = (mm >> lane) & 1u;
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    if (a >= naggs) break;
                    const int64_t x = warp_sum(in ? v[a][i] : int64_t(0));
                    if (lane == 0) v[a][i] = x;
                }
                if (in && lane != 0) apply = 0xffffffffu;
            }
            if (apply == 0xffffffffu) continue;
            if (SHARED) {
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    if (a >= naggs) break;
                    const size_t o = static_cast<size_t>(a) * f.D + apply;
                    add_split(&s_lo[o], &s_hi[o], static_cast<uint64_t>(v[a][i]));
                }
                if (f.count_agg < 0) red_or_shared(&s_occ[apply / 32], 1u << (apply % 32));
            } else {
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    if (a >= naggs) break;
                    red_add_global(&f.acc[static_cast<size_t>(a) * f.D + apply], static_cast<unsigned long long>(v[a][i]));
                }
                if (f.count_agg < 0) f.occ[apply] = 1;  // every writer stores the same value
            }
        }
    }
}

// Persistent fused kernel: (fragment, chunk) work items from a device counter.
template <int THREADS, int ITEMS, int NA>
__global__ void __launch_bounds__(THREADS)
frag_kernel(const PlanHeader* __restrict__ ph, const int64_t* __restrict__ item_start, const FragDev* __restrict__ fd,
            unsigned long long* counter, int32_t* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t s_item;
    __shared__ int32_t s_p;
    // The work item's fragment plan, copied to shared memory once per item: the
    // reductions' memory clobbers would otherwise reload its fields from global
    // memory after every update.
    __shared__ __align__(16) FragDev s_f;
    const int n = ph->nfrags;
    const int64_t nitems = ph->nitems;
    for (;;) {
        if (threadIdx.x == 0) {
            const int64_t it = static_cast<int64_t>(atomicAdd(counter, 1ull));
            s_item = it;
            s_p = it < nitems ? find_frag(item_start, n, it) : 0;
        }
        __syncthreads();
        const int64_t item = s_item;
        const int p = s_p;
        if (item < nitems) {
            const uint32_t* src = reinterpret_cast<const uint32_t*>(&fd[p]);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&s_f);
            for (int w = threadIdx.x; w < static_cast<int>(sizeof(FragDev) / 4); w += THREADS) dst[w] = src[w];
        }
        __syncthreads();
        if (item >= nitems) break;
        const FragDev& f = s_f;
        // A table this fragment cannot use: its rows are skipped.
        if (f.t.hdr->magic != kMagic || f.t.hdr->nsegs != 1 || f.t.hdr->unique == 0 || f.t.hdr->nbuild > f.nbuild) {
            if (threadIdx.x == 0) set_status(status, PX_ERR_INVALID);
            continue;
        }
        const int64_t r0 = (item - item_start[p]) * f.chunk;
        const int64_t r1 = r0 + f.chunk < f.nrows ? r0 + f.chunk : f.nrows;
        if (!f.shared) {
            frag_rows<THREADS, ITEMS, NA, false>(f, r0, r1, nullptr, nullptr, nullptr, status);
            continue;
        }
        const uint32_t D = f.D;
        const int naggs = f.naggs;
        uint32_t* s_lo = reinterpret_cast<uint32_t*>(smem);
        uint32_t* s_hi = s_lo + static_cast<size_t>(naggs) * D;
        uint32_t* s_occ = s_hi + static_cast<size_t>(naggs) * D;
        const uint32_t words = 2 * naggs * D + (f.count_agg < 0 ? (D + 31) / 32 : 0);
        for (uint32_t w = threadIdx.x; w < words; w += THREADS) s_lo[w] = 0;
        __syncthreads();
        frag_rows<THREADS, ITEMS, NA, true>(f, r0, r1, s_lo, s_hi, s_occ, status);
        __syncthreads();
        for (uint32_t d = threadIdx.x; d < D; d += THREADS) {
            bool occ = f.count_agg < 0 && ((s_occ[d / 32] >> (d % 32)) & 1u);
            for (int a = 0; a < naggs; ++a) {
                const size_t o = static_cast<size_t>(a) * D + d;
                const uint64_t x = (static_cast<uint64_t>(s_hi[o]) << 32) | s_lo[o];
                if (x) red_add_global(&f.acc[o], x);
                if (a == f.count_agg) occ = x != 0;
            }
            if (occ && f.count_agg < 0) f.occ[d] = 1;
        }
        // The next item's clear waits for every thread's flush at the loop top.
    }
}

// Writes each fragment's occupied slots as output groups in key order.
__global__ void __launch_bounds__(kEmitThreads)
frag_emit_kernel(const PlanHeader* __restrict__ ph, const int64_t* __restrict__ emit_start,
                 const FragDev* __restrict__ fd, unsigned long long* counter, int32_t* status) {
    __shared__ int64_t s_tile;
    __shared__ int64_t s_excl;
    __shared__ int32_t s_warp[kEmitThreads / 32];
    const int64_t tile = next_tile(counter, &s_tile);
    const int p = find_frag(emit_start, ph->nfrags, tile);
    const FragDev& f = fd[p];
    const int64_t lt = tile - emit_start[p];  // tile within the fragment
    const int64_t ntiles = emit_start[p + 1] - emit_start[p];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = lt * kEmitTile + warp * (32 * kEmitItems);
    const int64_t D = f.D;
    uint32_t mask[kEmitItems];
    int32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < kEmitItems; ++i) {
        const int64_t e = base + i * 32 + lane;
        bool occ = false;
        if (e < D) occ = f.count_agg >= 0 ? f.acc[f.count_agg * D + e] != 0 : f.occ[e] != 0;
        mask[i] = __ballot_sync(FULL, occ);
        cnt += __popc(mask[i]);
    }
    if (lane == 0) s_warp[warp] = cnt;
    __syncthreads();
    if (warp == 0) {
        const int32_t w = lane < kEmitThreads / 32 ? s_warp[lane] : 0;
        const int32_t incl = warp_incl_scan(w);
        const int32_t total = __shfl_sync(FULL, incl, 31);
        if (lane < kEmitThreads / 32) s_warp[lane] = incl - w;
        const int64_t excl = lookback(f.emit_states, lt, total, status);
        if (lane == 0) {
            s_excl = excl;
            if (lt == ntiles - 1) {
                *f.ngroups = excl + total;
                if (excl + total > f.max_groups) set_status(status, PX_ERR_CAPACITY);
            }
        }
    }
    __syncthreads();
    int64_t pos = s_excl + s_warp[warp];
    const uint32_t ltm = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kEmitItems; ++i) {
        if (mask[i] & (1u << lane)) {
            const int64_t e = base + i * 32 + lane;
            const int64_t q = pos + __popc(mask[i] & ltm);
            if (q < f.max_groups) {
                store_int(f.out_keys, f.group_w, q, f.group_lo + e);
                for (int a = 0; a < f.naggs; ++a) f.out_aggs[a][q] = static_cast<int64_t>(f.acc[a * D + e]);
            }
        }
        pos += __popc(mask[i]);
    }
}

bool valid_type(int32_t t) { return t == PX_I8 || t == PX_I32 || t == PX_I64; }

struct WsLayout {
    size_t counters, plan, acc, states, total;
};

// Accumulator bytes of fragment f: naggs x D 64-bit words, then D occupancy flags
// when there is no COUNT (256-byte aligned).
size_t frag_acc_bytes(const px_fragment& f) {
    const uint64_t D = static_cast<uint64_t>(f.group_hi - f.group_lo) + 1;
    bool has_count = false;
    for (int a = 0; a < f.naggs; ++a) has_count |= f.aggs[a].op == PX_COUNT;
    return align_up(8 * static_cast<size_t>(f.naggs) * D + (has_count ? 0 : D), 256);
}
size_t frag_state_bytes(const px_fragment& f) {
    const int64_t D = f.group_hi - f.group_lo + 1;
    return align_up(8 * static_cast<size_t>(cdiv(D, kEmitTile)), 256);
}

WsLayout frag_ws_layout(const px_fragment* frags, int32_t n) {
    WsLayout L;
    L.counters = kWsScratch;
    L.plan = L.counters + 256;
    L.acc = L.plan + align_up(plan_layout(n).total, 256);
    size_t acc = 0, st = 0;
    for (int32_t i = 0; i < n; ++i) {
        acc += frag_acc_bytes(frags[i]);
        st += frag_state_bytes(frags[i]);
    }
    L.states = L.acc + acc;
    L.total = L.states + st;
    return L;
}

px_status check_fragment(const px_fragment& f, int32_t i) {
    if (f.nrows < 0 || f.nrows > INT32_MAX) return fail(PX_ERR_INVALID, "px_fragments_run: fragment %d nrows", i);
    if (f.key.type != PX_I64 || (f.nrows > 0 && (!f.key.data || !aligned16(f.key.data))))
        return fail(PX_ERR_INVALID, "px_fragments_run: fragment %d key must be an aligned PX_I64 column", i);
    if (f.filter.data && (!valid_type(f.filter.type) || !aligned16(f.filter.data)))
        return fail(PX_ERR_INVALID, "px_fragments_run: fragment %d filter column", i);
    if (f.ncols < 0 || f.ncols > PX_FRAG_MAX_COLS || f.naggs < 0 || f.naggs > PX_FRAG_MAX_AGGS)
        return fail(PX_ERR_UNSUPPORTED, "px_fragments_run: fragment %d has %d columns, %d aggregates", i, f.ncols,
                    f.naggs);
    for (int c = 0; c < f.ncols; ++c)
        if (!valid_type(f.cols[c].type) || (f.nrows > 0 && (!f.cols[c].data || !aligned16(f.cols[c].data))))
            return fail(PX_ERR_INVALID, "px_fragments_run: fragment %d column %d", i, c);
    for (int a = 0; a < f.naggs; ++a) {
        const px_agg& g = f.aggs[a];
        if (g.op != PX_COUNT && g.op != PX_SUM && g.op != PX_SUM_MUL)
            return fail(PX_ERR_INVALID, "px_fragments_run: fragment %d aggregate %d op %d", i, a, g.op);
        if (g.op != PX_COUNT && (g.a < 0 || g.a >= f.ncols))
            return fail(PX_ERR_INVALID, "px_fragments_run: fragment %d aggregate %d column a", i, a);
        if (g.op == PX_SUM_MUL && (g.b < 0 || g.b >= f.ncols))
            return fail(PX_ERR_INVALID, "px_fragments_run: fragment %d aggregate %d column b", i, a);
        if (f.max_groups > 0 && !f.d_out_aggs[a])
            return fail(PX_ERR_INVALID, "px_fragments_run: fragment %d null output aggregate %d", i, a);
    }
    if (!f.d_table || !aligned16(f.d_table)) return fail(PX_ERR_INVALID, "px_fragments_run: fragment %d table", i);
    if (f.nbuild < 0 || !valid_type(f.group.type) || (f.nbuild > 0 && !f.group.data))
        return fail(PX_ERR_INVALID, "px_fragments_run: fragment %d group column", i);
    if (f.group_hi < f.group_lo ||
        static_cast<uint64_t>(f.group_hi) - static_cast<uint64_t>(f.group_lo) >= static_cast<uint64_t>(PX_FRAG_MAX_GROUPS))
        return fail(PX_ERR_UNSUPPORTED, "px_fragments_run: fragment %d group range [%lld, %lld]", i,
                    (long long)f.group_lo, (long long)f.group_hi);
    if (f.max_groups < 0 || (f.max_groups > 0 && !f.d_out_keys) || !f.d_ngroups)
        return fail(PX_ERR_INVALID, "px_fragments_run: fragment %d outputs", i);
    return PX_OK;
}

template <int THREADS, int ITEMS, int NA>
px_status launch_frag_na(const PlanHeader* ph, const int64_t* item_start, const FragDev* fd,
                         unsigned long long* counter, int32_t* status, size_t smem, int bps, cudaStream_t st) {
    auto kernel = frag_kernel<THREADS, ITEMS, NA>;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
        cudaSuccess)
        return check_launch("px_fragments_run attribute");
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, THREADS, smem);
    if (per_sm < 1) return fail(PX_ERR_UNSUPPORTED, "px_fragments_run: configuration does not fit an SM");
    const int blocks = sm_count() * std::min(per_sm, bps);
    kernel<<<blocks, THREADS, smem, st>>>(ph, item_start, fd, counter, status);
    note_launch();
    return check_launch("px_fragments_run fused");
}

// NA: the batch's largest aggregate count (at least 1), a compile-time bound.
template <int THREADS, int ITEMS>
px_status launch_frag(int na, const PlanHeader* ph, const int64_t* item_start, const FragDev* fd,
                      unsigned long long* counter, int32_t* status, size_t smem, int bps, cudaStream_t st) {
    switch (na) {
        case 0:
        case 1: return launch_frag_na<THREADS, ITEMS, 1>(ph, item_start, fd, counter, status, smem, bps, st);
        case 2: return launch_frag_na<THREADS, ITEMS, 2>(ph, item_start, fd, counter, status, smem, bps, st);
        case 3: return launch_frag_na<THREADS, ITEMS, 3>(ph, item_start, fd, counter, status, smem, bps, st);
        default: return launch_frag_na<THREADS, ITEMS, 4>(ph, item_start, fd, counter, status, smem, bps, st);
    }
}

}  // namespace
}  // namespace px

using namespace px;

extern "C" {

size_t px_fragments_plan_bytes(int32_t nfrags) { return plan_layout(nfrags < 0 ? 0 : nfrags).total; }

size_t px_fragments_ws_bytes(const px_fragment* frags, int32_t nfrags) {
    if (!frags || nfrags < 0) return kWsScratch + 256;
    return frag_ws_layout(frags, nfrags).total;
}

px_status px_fragments_run(const px_fragment* frags, int32_t nfrags, const px_fragments_config* cfg, void* h_plan,
                           size_t plan_bytes, void* d_ws, size_t ws_bytes, void* stream) {
    CallRange nvtx_range("px_fragments_run");
    set_error("");
    if (nfrags < 0 || (nfrags > 0 && !frags)) return fail(PX_ERR_INVALID, "px_fragments_run: bad fragment list");
    if (nfrags > INT32_MAX / 2) return fail(PX_ERR_UNSUPPORTED, "px_fragments_run: too many fragments");
    for (int32_t i = 0; i < nfrags; ++i) {
        const px_status s = check_fragment(frags[i], i);
        if (s != PX_OK) return s;
    }
    px_fragments_config c = {256, 2, 0, 8};
    if (cfg) c = *cfg;
    if ((c.threads != 256 && c.threads != 512) || (c.items != 2 && c.items != 4) || c.blocks_per_sm < 1 ||
        c.blocks_per_sm > 8 || c.chunk_rows < 0 || c.chunk_rows % (static_cast<int64_t>(c.threads) * c.items) != 0)
        return fail(PX_ERR_INVALID, "px_fragments_run: bad configuration");
    if (c.chunk_rows == 0) {
        // Rows per work item from the batch: about four items per block of the
        // persistent grid, so a small batch still spreads over every SM, within
        // [one tile, 65536 rows].
        const int64_t tile = static_cast<int64_t>(c.threads) * c.items;
        int64_t rows = 0;
        for (int32_t i = 0; i < nfrags; ++i) rows += frags[i].nrows;
        const int64_t want = cdiv(rows, 4 * static_cast<int64_t>(sm_count()) * c.blocks_per_sm);
        c.chunk_rows = std::min<int64_t>(std::max<int64_t>(cdiv(want, tile) * tile, tile), cdiv(65536, tile) * tile);
    }
    const PlanLayout PL = plan_layout(nfrags);
    if (!h_plan || plan_bytes < PL.total)
        return fail(PX_ERR_INVALID, "px_fragments_run: plan staging of %zu bytes, %zu needed", plan_bytes, PL.total);
    const WsLayout L = frag_ws_layout(frags, nfrags);
    px_status s = check_ws(d_ws, ws_bytes, L.total, "px_fragments_run");
    if (s != PX_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (nfrags == 0) return PX_OK;

    // Work order: decreasing fragment size, so the longest fragments start first.
    std::vector<int32_t> order(nfrags);
    for (int32_t i = 0; i < nfrags; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t x, int32_t y) { return frags[x].nrows > frags[y].nrows; });

    char* hp = static_cast<char*>(h_plan);
    PlanHeader* ph = reinterpret_cast<PlanHeader*>(hp);
    int64_t* item_start = reinterpret_cast<int64_t*>(hp + PL.items);
    int64_t* emit_start = reinterpret_cast<int64_t*>(hp + PL.emits);
    FragDev* fd = reinterpret_cast<FragDev*>(hp + PL.frags);
    char* ws = static_cast<char*>(d_ws);
    const int64_t tile = static_cast<int64_t>(c.threads) * c.items;
    // Accumulator and emit-state areas are laid out in the caller's order.
    std::vector<size_t> acc_off(nfrags), st_off(nfrags);
    size_t acc = 0, sto = 0;
    for (int32_t i = 0; i < nfrags; ++i) {
        acc_off[i] = acc;
        st_off[i] = sto;
        acc += frag_acc_bytes(frags[i]);
        sto += frag_state_bytes(frags[i]);
    }
    size_t smem = 0;
    int64_t items = 0, emits = 0;
    for (int32_t k = 0; k < nfrags; ++k) {
        const int32_t i = order[k];
        const px_fragment& f = frags[i];
        FragDev& d = fd[k];
        d = FragDev{};
        d.key = static_cast<const int64_t*>(f.key.data);
        d.filter = f.filter.data;
        d.filter_w = f.filter.type;
        d.lo = f.lo;
        d.hi = f.hi;
        d.nrows = f.nrows;
        d.naggs = f.naggs;
        d.count_agg = -1;
        for (int a = 0; a < f.naggs; ++a) {
            const px_agg& g = f.aggs[a];
            d.op[a] = g.op;
            if (g.op != PX_COUNT) {
                d.pa[a] = f.cols[g.a].data;
                d.wa[a] = f.cols[g.a].type;
            }
            if (g.op == PX_SUM_MUL) {
                d.pb[a] = f.cols[g.b].data;
                d.wb[a] = f.cols[g.b].type;
            }
            if (g.op == PX_COUNT && d.count_agg < 0) d.count_agg = a;
        }
        d.t = table_view(const_cast<void*>(f.d_table), 1);
        d.nbuild = f.nbuild;
        d.group = f.group.data;
        d.group_w = f.group.type;
        d.group_lo = f.group_lo;
        d.D = static_cast<uint32_t>(f.group_hi - f.group_lo + 1);
        // Shared mode when the block arrays fit and a work item can be at least 4 D
        // rows (so clearing and flushing them stays a small part of the item).
        const size_t sbytes = 8 * static_cast<size_t>(f.naggs) * d.D + (d.count_agg < 0 ? (d.D + 31) / 32 * 4 : 0);
        d.shared = sbytes <= kSmemAccBudget && f.nrows >= 4 * static_cast<int64_t>(d.D) ? 1 : 0;
        d.chunk = c.chunk_rows;
        if (d.shared) {
            d.chunk = std::max<int64_t>(c.chunk_rows, cdiv(4 * static_cast<int64_t>(d.D), tile) * tile);
            smem = std::max(smem, sbytes);
        }
        d.acc = reinterpret_cast<unsigned long long*>(ws + L.acc + acc_off[i]);
        d.occ = d.count_agg < 0 ? reinterpret_cast<uint8_t*>(ws + L.acc + acc_off[i]) + 8 * static_cast<size_t>(f.naggs) * d.D
                                : nullptr;
        d.emit_states = reinterpret_cast<uint64_t*>(ws + L.states + st_off[i]);
        d.out_keys = f.d_out_keys;
        for (int a = 0; a < f.naggs; ++a) d.out_aggs[a] = f.d_out_aggs[a];
        d.ngroups = f.d_ngroups;
        d.max_groups = f.max_groups;
        item_start[k] = items;
        emit_start[k] = emits;
        items += cdiv(f.nrows, d.chunk);
        emits += cdiv(static_cast<int64_t>(d.D), kEmitTile);
    }
    item_start[nfrags] = items;
    emit_start[nfrags] = emits;
    *ph = PlanHeader{};
    ph->nfrags = nfrags;
    ph->nitems = items;
    ph->nemit = emits;

    char* dplan = ws + L.plan;
    unsigned long long* counters = reinterpret_cast<unsigned long long*>(ws + L.counters);
    int32_t* status = &static_cast<WsHeader*>(d_ws)->status;
    cudaMemsetAsync(counters, 0, 256, st);
    cudaMemsetAsync(ws + L.acc, 0, L.total - L.acc, st);
    cudaMemcpyAsync(dplan, h_plan, PL.total, cudaMemcpyHostToDevice, st);
    const PlanHeader* d_ph = reinterpret_cast<const PlanHeader*>(dplan);
    const int64_t* d_items = reinterpret_cast<const int64_t*>(dplan + PL.items);
    const int64_t* d_emits = reinterpret_cast<const int64_t*>(dplan + PL.emits);
    const FragDev* d_fd = reinterpret_cast<const FragDev*>(dplan + PL.frags);
    if (items > 0) {
        int na = 0;
        for (int32_t i = 0; i < nfrags; ++i) na = std::max(na, frags[i].naggs);
        if (c.threads == 256 && c.items == 2)
            s = launch_frag<256, 2>(na, d_ph, d_items, d_fd, counters, status, smem, c.blocks_per_sm, st);
        else if (c.threads == 256)
            s = launch_frag<256, 4>(na, d_ph, d_items, d_fd, counters, status, smem, c.blocks_per_sm, st);
        else if (c.items == 2)
            s = launch_frag<512, 2>(na, d_ph, d_items, d_fd, counters, status, smem, c.blocks_per_sm, st);
        else
            s = launch_frag<512, 4>(na, d_ph, d_items, d_fd, counters, status, smem, c.blocks_per_sm, st);
        if (s != PX_OK) return s;
    }
    frag_emit_kernel<<<static_cast<unsigned>(emits), kEmitThreads, 0, st>>>(d_ph, d_emits, d_fd, counters + 1, status);
    note_launch();
    return check_launch("px_fragments_run emit");
}

}  // extern "C"
