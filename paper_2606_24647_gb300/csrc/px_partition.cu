// px_partition: PartitionedOutput's hash partitioning (Sec. 3.1, Sec. 3.3.2) as an
// on-device exchange. The output is one packed buffer per column holding partition
// 0's rows, then partition 1's, ... (stable), plus offsets[nparts+1]: the
// UcxExchange's "size metadata, then packed GPU data" for every destination.
//
// Three launches over tiles of T positions (T = 512, 1024 or 2048, chosen so a
// tile of every column fits the shared-memory staging area):
//   1. hist    - per-tile partition counts, stored partition-major: cnt[q][t]
//                (per-warp shared counters, native 32-bit atomics).
//   2. scan    - exclusive scan of cnt in that order gives each (partition, tile)
//                its global output start (single pass, bounded look-back), and
//                offsets[q] = start of (q, tile 0).
//   3. scatter - stages the tile of every column into shared memory with one TMA
//                bulk copy per column (all in flight together, completed on an
//                mbarrier; plain loads for gathers through a selection and for a
//                ragged last tile), ranks rows stably inside the tile with a warp
//                multi-split (one ballot per partition-id bit gives the lanes with
//                the same partition) and per-warp counters, then per column moves
//                the values into partition order in shared memory and writes each
//                partition's run contiguously, so the stores coalesce.
// The key column is read twice (hist and scatter); every other column once; every
// column written once.
#include <algorithm>
#include <type_traits>

#include "px_common.cuh"

namespace px {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr size_t kStageBudget = 48 * 1024;  // raw tile staging bytes (all columns)
constexpr int kOffRegs = (PX_MAX_PARTS + kThreads - 1) / kThreads;  // partitions per thread, at most

constexpr int kScanThreads = 256;
constexpr int kScanItems = 32;  // 8192 counts per scan tile: a short look-back chain
constexpr int kScanTile = kScanThreads * kScanItems;
// Up to this many partitions the histogram pass stores each position's partition id
// (one byte) for the scatter, which then stages the ids instead of hashing the keys
// again: one byte written and read per row against a hash per row.
constexpr int32_t kPidMaxParts = 256;

struct Cols {
    int32_t ncols;
    int32_t width[PX_MAX_COLS];
    const void* in[PX_MAX_COLS];
    void* out[PX_MAX_COLS];
    uint32_t stage_off[PX_MAX_COLS];  // byte offset of the column's tile in the staging area
    int32_t order[PX_MAX_COLS];       // columns by decreasing width (the order they are moved in)
};

// Items per thread so that the staged tile of all columns fits kStageBudget.
int items_for(int64_t row_bytes) {
    if (row_bytes * kThreads * 8 <= static_cast<int64_t>(kStageBudget)) return 8;
    if (row_bytes * kThreads * 4 <= static_cast<int64_t>(kStageBudget)) return 4;
    return 2;
}

// Local position of item i of this thread inside a tile: warp-contiguous runs of
// 32 * ITEMS positions, lanes innermost, so position order = (warp, item, lane).
template <int ITEMS>
__device__ __forceinline__ int local_pos(int warp, int i, int lane) {
    return warp * (32 * ITEMS) + i * 32 + lane;
}

template <int ITEMS>
__global__ void __launch_bounds__(kThreads)
part_hist_kernel(const int64_t* __restrict__ key, const int32_t* __restrict__ sel,
                 const int64_t* __restrict__ d_nsel, int64_t ncap, uint64_t seed, uint32_t nparts,
                 int32_t* __restrict__ cnt, int64_t ntiles, uint8_t* __restrict__ pid_out) {
    constexpr int T = kThreads * ITEMS;
    extern __shared__ int32_t s_hist[];  // [kWarps][nparts]
    allow_dependents();  // the scan may launch now; it waits for this grid's counts
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (uint32_t q = tid; q < kWarps * nparts; q += kThreads) s_hist[q] = 0;
    const int64_t n = actual_rows(d_nsel, ncap);
    const int64_t tbase = static_cast<int64_t>(blockIdx.x) * T;
    uint32_t p[ITEMS];
    if (!sel && tbase + T <= n && (reinterpret_cast<uintptr_t>(key) & 15) == 0) {
        // A full tile of a plain column: only counts matter here, so each thread
        // takes ITEMS consecutive keys with 16-byte loads.
        const longlong2* kv = reinterpret_cast<const longlong2*>(key + tbase + static_cast<int64_t>(tid) * ITEMS);
#pragma unroll
        for (int i = 0; i < ITEMS / 2; ++i) {
            const longlong2 k2 = kv[i];
            p[2 * i] = part_of(k2.x, seed, nparts);
            p[2 * i + 1] = part_of(k2.y, seed, nparts);
        }
        if (pid_out) {  // the ids of this thread's ITEMS consecutive positions, one store
            uint64_t w = 0;
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) w |= static_cast<uint64_t>(p[i]) << (8 * i);
            uint8_t* o = pid_out + tbase + static_cast<int64_t>(tid) * ITEMS;
            if (ITEMS == 8) *reinterpret_cast<uint64_t*>(o) = w;
            else if (ITEMS == 4) *reinterpret_cast<uint32_t*>(o) = static_cast<uint32_t>(w);
            else *reinterpret_cast<uint16_t*>(o) = static_cast<uint16_t>(w);
        }
    } else {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const int64_t j = tbase + local_pos<ITEMS>(warp, i, lane);
            p[i] = nparts;
            if (j < n) {
                p[i] = part_of(key[sel ? static_cast<int64_t>(sel[j]) : j], seed, nparts);
                if (pid_out) pid_out[j] = static_cast<uint8_t>(p[i]);
            }
        }
    }
    __syncthreads();
    int32_t* wh = s_hist + warp * nparts;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
        if (p[i] < nparts) atomicAdd(&wh[p[i]], 1);
    __syncthreads();
    for (uint32_t q = tid; q < nparts; q += kThreads) {
        int32_t c = 0;
        for (int w = 0; w < kWarps; ++w) c += s_hist[w * nparts + q];
        cnt[static_cast<int64_t>(q) * ntiles + blockIdx.x] = c;
    }
}

// Exclusive scan of cnt[0..total) (partition-major) into offs; offsets[q] is the
// scanned value at (q, tile 0) and offsets[nparts] the grand total.
__global__ void __launch_bounds__(kScanThreads)
part_scan_kernel(const int32_t* __restrict__ cnt, int32_t* __restrict__ offs, int64_t total,
                 int64_t ntiles, uint32_t nparts, int64_t* __restrict__ d_offsets, ScanScratch scan,
                 int32_t* status, int64_t nscan_tiles) {
    __shared__ int64_t s_tile;
    __shared__ int32_t s_warp[33];
    __shared__ int64_t s_excl;
    wait_prior();        // the histogram's counts (and its partition ids) are complete
    allow_dependents();  // so the scatter, launched from here on, may read those ids at once
    const int64_t tile = next_tile(scan.counter, &s_tile);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = tile * kScanTile + static_cast<int64_t>(tid) * kScanItems;
    int32_t v[kScanItems];
    int32_t sum = 0;
    const bool full = base + kScanItems <= total;  // a thread's run is 128-byte aligned
    if (full) {
#pragma unroll
        for (int k = 0; k < kScanItems; k += 4) {
            const int4 x = *reinterpret_cast<const int4*>(cnt + base + k);
            v[k] = x.x;
            v[k + 1] = x.y;
            v[k + 2] = x.z;
            v[k + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) v[k] = base + k < total ? cnt[base + k] : 0;
    }
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) sum += v[k];
    const int32_t incl = warp_incl_scan(sum);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int32_t w = lane < kScanThreads / 32 ? s_warp[lane] : 0;
        const int32_t wi = warp_incl_scan(w);
        if (lane < kScanThreads / 32) s_warp[lane] = wi - w;
        const int32_t agg = __shfl_sync(FULL, wi, 31);
        const int64_t excl = lookback(scan.states, tile, agg, status);
        if (lane == 0) {
            s_excl = excl;
            if (tile == nscan_tiles - 1) d_offsets[nparts] = excl + agg;
        }
    }
    __syncthreads();
    int64_t run = s_excl + s_warp[warp] + incl - sum;
    // Partition starts inside this thread's run: the multiples of ntiles there.
    int64_t next_q = (base + ntiles - 1) / ntiles;  // first partition starting at or after base
    int64_t next_e = next_q * ntiles;
    int32_t o[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t e = base + k;
        o[k] = static_cast<int32_t>(run);
        if (e < total && e == next_e) {
            d_offsets[next_q] = run;
            ++next_q;
            next_e += ntiles;
        }
        run += v[k];
    }
    if (full) {
#pragma unroll
        for (int k = 0; k < kScanItems; k += 4)
            *reinterpret_cast<int4*>(offs + base + k) = make_int4(o[k], o[k + 1], o[k + 2], o[k + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k)
            if (base + k < total) offs[base + k] = o[k];
    }
}

// Moves one column's tile from the staging area (tile order) into partition order
// in buffer `buf` (shared memory).
// FT: a full tile, where every position holds a row (no per-row checks).
template <typename T, int ITEMS, bool FT>
__device__ __forceinline__ void transpose_col(const unsigned char* staged, unsigned char* buf, const int32_t* posv,
                                              const uint32_t* pidv, uint32_t nparts, int warp, int lane) {
    const T* src = reinterpret_cast<const T*>(staged);
    T* sorted = reinterpret_cast<T*>(buf);
    T v[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
        if (FT || pidv[i] < nparts) v[i] = src[local_pos<ITEMS>(warp, i, lane)];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
        if (FT || pidv[i] < nparts) sorted[posv[i]] = v[i];
}

// Writes a partition-ordered column tile to its global rows: dest[k] is the output
// row of partition-ordered position threadIdx.x + k * kThreads (-1 past the tile),
// so each partition's run is written contiguously.
template <typename T, int ITEMS, bool FT>
__device__ __forceinline__ void store_col(const unsigned char* buf, const int32_t* dest, void* out) {
    const T* sorted = reinterpret_cast<const T*>(buf);
    T* o = static_cast<T*>(out);
#pragma unroll
    for (int k = 0; k < ITEMS; ++k)
        if (FT || dest[k] >= 0) o[dest[k]] = sorted[threadIdx.x + k * kThreads];
}

template <typename T, int ITEMS>
__device__ __forceinline__ void stage_plain(const T* in, T* staged, const int32_t* __restrict__ sel, int64_t tbase,
                                            int tile_rows, int warp, int lane) {
    T v[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int lp = local_pos<ITEMS>(warp, i, lane);
        const int64_t j = tbase + lp;
        if (lp < tile_rows) v[i] = in[sel ? static_cast<int64_t>(sel[j]) : j];
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int lp = local_pos<ITEMS>(warp, i, lane);
        if (lp < tile_rows) staged[lp] = v[i];
    }
}

// NBITS: bits of the largest partition id (nparts - 1), so the multi-split below
// is unrolled: one ballot per id bit, plus one for the valid rows of a ragged tile.
template <int ITEMS, int NBITS>
__global__ void __launch_bounds__(kThreads, ITEMS >= 8 ? 3 : 4)
part_scatter_kernel(Cols cols, int32_t key_col, const int32_t* __restrict__ sel,
                    const int64_t* __restrict__ d_nsel, int64_t ncap, uint64_t seed, uint32_t nparts,
                    const int32_t* __restrict__ offs, int64_t ntiles, uint32_t stage_bytes, uint32_t row_bytes,
                    const uint8_t* __restrict__ pid_in, int32_t* status) {
    constexpr int T = kThreads * ITEMS;
    extern __shared__ __align__(16) unsigned char smem[];
    const int np1 = static_cast<int>(nparts) + 1;
    const int np1p = (np1 + 3) & ~3;
    unsigned char* stage = smem;                                                   // stage_bytes
    void* sorted = smem + stage_bytes;                                             // T x 8 B
    int32_t* s_dest = reinterpret_cast<int32_t*>(smem + stage_bytes + T * 8);     // T
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + stage_bytes + T * 12);     // 16 B
    int32_t* s_delta = reinterpret_cast<int32_t*>(smem + stage_bytes + T * 12 + 16);  // np1p
    int32_t* s_whist = s_delta + np1p;                                             // kWarps x np1
    // partition ids from the histogram pass (T bytes), when it wrote them
    uint8_t* s_pid = smem + ((stage_bytes + T * 12 + 16 + (np1p + kWarps * np1) * 4 + 15) & ~15u);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t tile = blockIdx.x;
    const int64_t n = actual_rows(d_nsel, ncap);
    const int64_t tbase = tile * T;
    const int64_t rem = n - tbase;
    const int tile_rows = rem <= 0 ? 0 : (rem < T ? static_cast<int>(rem) : T);
    for (int k = tid; k < kWarps * np1; k += kThreads) s_whist[k] = 0;

    // Stage the tile of every column: TMA bulk copies for a full contiguous tile,
    // plain loads for a gather through a selection or a ragged last tile. The
    // columns are inputs of earlier calls: their copies start before the wait for
    // the scan (this kernel may be running while the scan finishes).
    const bool bulk = sel == nullptr && tile_rows == T;
    if (bulk) {
        if (tid == 0) {
            mbar_init(bar, 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (tid == 0) {
            mbar_arrive_expect_tx(bar, static_cast<uint32_t>(T) * (row_bytes + (pid_in ? 1 : 0)));
            for (int c = 0; c < cols.ncols; ++c)
                bulk_g2s(stage + cols.stage_off[c], static_cast<const char*>(cols.in[c]) + tbase * cols.width[c],
                         static_cast<uint32_t>(T * cols.width[c]), bar);
        }
    }
    wait_prior();  // the scan's offsets, and the histogram's ids before it
    // This tile's output start in each partition (one strided load per partition),
    // requested now so its latency hides behind the staging of the tile.
    int32_t my_off[kOffRegs];
#pragma unroll
    for (int r = 0; r < kOffRegs; ++r) {
        const int q = tid + r * kThreads;
        my_off[r] = q < static_cast<int>(nparts) ? offs[static_cast<int64_t>(q) * ntiles + tile] : 0;
    }
    if (bulk) {
        if (tid == 0 && pid_in) bulk_g2s(s_pid, pid_in + tbase, static_cast<uint32_t>(T), bar);
        if (!mbar_wait(bar, 0) && lane == 0) set_status(status, PX_ERR_TIMEOUT);
    } else {
        for (int c = 0; c < cols.ncols; ++c) {
            unsigned char* st = stage + cols.stage_off[c];
            if (cols.width[c] == 8)
                stage_plain<int64_t, ITEMS>(static_cast<const int64_t*>(cols.in[c]), reinterpret_cast<int64_t*>(st),
                                            sel, tbase, tile_rows, warp, lane);
            else if (cols.width[c] == 4)
                stage_plain<int32_t, ITEMS>(static_cast<const int32_t*>(cols.in[c]), reinterpret_cast<int32_t*>(st),
                                            sel, tbase, tile_rows, warp, lane);
            else
                stage_plain<int8_t, ITEMS>(static_cast<const int8_t*>(cols.in[c]), reinterpret_cast<int8_t*>(st), sel,
                                           tbase, tile_rows, warp, lane);
        }
        if (pid_in)  // ids are stored by position, not through the selection
            stage_plain<uint8_t, ITEMS>(pid_in, s_pid, nullptr, tbase, tile_rows, warp, lane);
        __syncthreads();
    }

    // The rest runs specialised for a full tile (every position a row) or not.
    auto finish = [&](auto full_tile) {
        constexpr bool FT = decltype(full_tile)::value;
        // Partition of every row, then its stable rank inside the warp's run: the lanes
        // with the same partition id come from one ballot per id bit (multi-split); a
        // per-warp counter row carries ranks across the thread's items.
        const int64_t* keys = reinterpret_cast<const int64_t*>(stage + cols.stage_off[key_col]);
        uint32_t pidv[ITEMS];
        int32_t posv[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const int lp = local_pos<ITEMS>(warp, i, lane);
            pidv[i] = FT || lp < tile_rows ? (pid_in ? static_cast<uint32_t>(s_pid[lp]) : part_of(keys[lp], seed, nparts))
                                           : nparts;
        }
        int32_t* wh = s_whist + warp * np1;
        const uint32_t lt = lanemask_lt();
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            // A row past a ragged tile's end has p = nparts and is in no valid row's
            // peer set; it never updates a counter (it is not its own peers' leader).
            const uint32_t p = pidv[i];
            uint32_t peers = FT ? FULL : __ballot_sync(FULL, p < nparts);
#pragma unroll
            for (int b = 0; b < NBITS; ++b) {
                const bool bit = (p >> b) & 1u;
                const uint32_t bal = __ballot_sync(FULL, bit);
                peers &= bit ? bal : ~bal;
            }
            const int32_t base = wh[p];
            __syncwarp();
            if (lane == __ffs(peers) - 1) wh[p] = base + __popc(peers);
            __syncwarp();
            posv[i] = base + __popc(peers & lt);
        }
#pragma unroll
        for (int r = 0; r < kOffRegs; ++r) {
            const int q = tid + r * kThreads;
            if (q < static_cast<int>(nparts)) s_delta[q] = my_off[r];
        }
        __syncthreads();
        // Warp 0, 32 partitions at a time: the start of each partition's run in the tile
        // (warp scan of the partitions' counts) plus each warp's start inside the run
        // (scan of the warps' counters) turn s_whist[w][q] into the tile position of
        // warp w's first row of partition q, and s_delta[q] into the shift from a tile
        // position in partition q's run to its output row.
        if (warp == 0) {
            int32_t carry = 0;
            for (int base = 0; base < static_cast<int>(nparts); base += 32) {
                const int q = base + lane;
                int32_t run = 0;
                if (q < static_cast<int>(nparts))
                    for (int w = 0; w < kWarps; ++w) run += s_whist[w * np1 + q];
                const int32_t incl = warp_incl_scan(run);
                if (q < static_cast<int>(nparts)) {
                    int32_t at = carry + incl - run;
                    s_delta[q] -= at;
                    for (int w = 0; w < kWarps; ++w) {
                        const int32_t c = s_whist[w * np1 + q];
                        s_whist[w * np1 + q] = at;
                        at += c;
                    }
                }
                carry += __shfl_sync(FULL, incl, 31);
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            if (FT || pidv[i] < nparts) {
                posv[i] += wh[pidv[i]];
                s_dest[posv[i]] = posv[i] + s_delta[pidv[i]];
            }
        }
        __syncthreads();
        int32_t dest[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const int jj = tid + k * kThreads;
            dest[k] = FT || jj < tile_rows ? s_dest[jj] : -1;
        }

        // Column phases, one barrier each: phase k writes column order[k-1] to global
        // memory from its partition-ordered buffer while moving column order[k] into
        // partition order. The first column's buffer is the sorted area; column
        // order[k]'s is the staging area of column order[k-1], free once that column
        // was moved and at least as large (decreasing widths).
        for (int k = 0; k <= cols.ncols; ++k) {
            if (k > 0) {
                const int c = cols.order[k - 1];
                const unsigned char* buf =
                    k == 1 ? static_cast<const unsigned char*>(sorted) : stage + cols.stage_off[cols.order[k - 2]];
                switch (cols.width[c]) {
                    case 8: store_col<int64_t, ITEMS, FT>(buf, dest, cols.out[c]); break;
                    case 4: store_col<int32_t, ITEMS, FT>(buf, dest, cols.out[c]); break;
                    default: store_col<int8_t, ITEMS, FT>(buf, dest, cols.out[c]); break;
                }
            }
            if (k < cols.ncols) {
                const int c = cols.order[k];
                unsigned char* buf = k == 0 ? static_cast<unsigned char*>(sorted) : stage + cols.stage_off[cols.order[k - 1]];
                const unsigned char* st = stage + cols.stage_off[c];
                switch (cols.width[c]) {
                    case 8: transpose_col<int64_t, ITEMS, FT>(st, buf, posv, pidv, nparts, warp, lane); break;
                    case 4: transpose_col<int32_t, ITEMS, FT>(st, buf, posv, pidv, nparts, warp, lane); break;
                    default: transpose_col<int8_t, ITEMS, FT>(st, buf, posv, pidv, nparts, warp, lane); break;
                }
            }
            __syncthreads();
        }
    };
    if (tile_rows == T) finish(std::true_type{});
    else finish(std::false_type{});
}

size_t scatter_smem_bytes(int items, uint32_t stage_bytes, int32_t nparts) {
    const size_t T = static_cast<size_t>(kThreads) * items;
    const size_t np1 = static_cast<size_t>(nparts) + 1;
    const size_t np1p = (np1 + 3) & ~static_cast<size_t>(3);
    return align_up(stage_bytes + T * 12 + 16 + np1p * 4 + kWarps * np1 * 4, size_t(16)) + T;  // + ids
}

// Workspace: count matrix, offset matrix (partition-major, P x tiles int32) and the
// scan scratch, sized for the smallest tile (2 items per thread).
struct PartScratch {
    int32_t* cnt;
    int32_t* offs;
    void* scan;
    size_t scan_bytes;
    uint8_t* pid;  // one partition id per position (nparts <= 256), or null
};

size_t part_mat_bytes(int64_t nrows, int32_t nparts) {
    return align_up(static_cast<size_t>(cdiv(nrows, kThreads * 2)) * nparts * 4, 256);
}

PartScratch part_scratch(void* d_ws, int64_t nrows, int64_t ntiles, int32_t nparts) {
    PartScratch p;
    char* base = static_cast<char*>(d_ws) + kWsScratch;
    const size_t mat = part_mat_bytes(nrows, nparts);
    p.cnt = reinterpret_cast<int32_t*>(base);
    p.offs = reinterpret_cast<int32_t*>(base + mat);
    p.scan = base + 2 * mat;
    p.scan_bytes = scan_scratch_bytes(cdiv(ntiles * nparts, kScanTile));
    p.pid = nparts <= kPidMaxParts ? reinterpret_cast<uint8_t*>(base + 2 * mat + p.scan_bytes) : nullptr;
    return p;
}

// blocks_per_sm > 0 caps the scatter's resident blocks per SM by asking each
// block for a larger share of the SM's shared memory than it needs (a launch
// shape the autotuner explores); 0 leaves residency to the kernel's own needs.
template <int ITEMS>
px_status launch_partition(const Cols& cols, int32_t key_col, const int32_t* d_sel, const int64_t* d_n, int64_t ncap,
                           uint64_t seed, int32_t nparts, int64_t* d_offsets, const PartScratch& ps, int64_t ntiles,
                           uint32_t stage_bytes, uint32_t row_bytes, int32_t blocks_per_sm, int32_t* status,
                           cudaStream_t st) {
    px_status s;
    const int64_t* key = static_cast<const int64_t*>(cols.in[key_col]);
    cudaMemsetAsync(ps.scan, 0, ps.scan_bytes, st);  // before the histogram: the scan launches right after it
    part_hist_kernel<ITEMS><<<static_cast<unsigned>(ntiles), kThreads, kWarps * nparts * sizeof(int32_t), st>>>(
        key, d_sel, d_n, ncap, seed, static_cast<uint32_t>(nparts), ps.cnt, ntiles, ps.pid);
    note_launch();
    if ((s = check_launch("px_partition hist")) != PX_OK) return s;

    const int64_t total = ntiles * nparts;
    const int64_t nscan = cdiv(total, kScanTile);
    launch_after(part_scan_kernel, dim3(static_cast<unsigned>(nscan)), dim3(kScanThreads), 0, st, ps.cnt, ps.offs, total,
                 ntiles, static_cast<uint32_t>(nparts), d_offsets, scan_scratch(ps.scan), status, nscan);
    note_launch();
    if ((s = check_launch("px_partition scan")) != PX_OK) return s;

    size_t smem = scatter_smem_bytes(ITEMS, stage_bytes, nparts);
    if (blocks_per_sm > 0) {
        int dev = 0, per_sm_smem = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        // each resident block also holds 1 KB the system reserves
        const size_t share = static_cast<size_t>(per_sm_smem) / blocks_per_sm;
        const size_t want = share > 1024 + 16 ? share - 1024 - 16 : 0;
        int max_block = 0;
        cudaDeviceGetAttribute(&max_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (want > smem) smem = std::min(want, static_cast<size_t>(max_block));
    }
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        launch_after(kern, dim3(static_cast<unsigned>(ntiles)), dim3(kThreads), smem, st, cols, key_col, d_sel, d_n,
                     ncap, seed, static_cast<uint32_t>(nparts), ps.offs, ntiles, stage_bytes, row_bytes, ps.pid,
                     status);
    };
    static_assert(PX_MAX_PARTS <= 1024, "partition ids need at most 10 bits");
    switch (nparts <= 1 ? 0 : 32 - __builtin_clz(static_cast<unsigned>(nparts - 1))) {
        case 0: go(part_scatter_kernel<ITEMS, 0>); break;
        case 1: go(part_scatter_kernel<ITEMS, 1>); break;
        case 2: go(part_scatter_kernel<ITEMS, 2>); break;
        case 3: go(part_scatter_kernel<ITEMS, 3>); break;
        case 4: go(part_scatter_kernel<ITEMS, 4>); break;
        case 5: go(part_scatter_kernel<ITEMS, 5>); break;
        case 6: go(part_scatter_kernel<ITEMS, 6>); break;
        case 7: go(part_scatter_kernel<ITEMS, 7>); break;
        case 8: go(part_scatter_kernel<ITEMS, 8>); break;
        case 9: go(part_scatter_kernel<ITEMS, 9>); break;
        default: go(part_scatter_kernel<ITEMS, 10>); break;
    }
    note_launch();
    return check_launch("px_partition scatter");
}

}  // namespace
}  // namespace px

using namespace px;

extern "C" {

size_t px_partition_ws_bytes(int64_t nrows, int32_t nparts) {
    if (nrows < 0) nrows = 0;
    if (nparts < 1) nparts = 1;
    const int64_t max_tiles = cdiv(nrows, kThreads * 2);
    return kWsScratch + 2 * part_mat_bytes(nrows, nparts) + scan_scratch_bytes(cdiv(max_tiles * nparts, kScanTile)) +
           (nparts <= kPidMaxParts ? align_up(static_cast<size_t>(nrows), 256) : 0);
}

px_status px_partition_tuned(const px_batch* in, int32_t key_col, const int32_t* d_sel, const int64_t* d_nsel,
                             int32_t nparts, uint64_t seed, const px_batch* out, int64_t* d_offsets,
                             const px_partition_config* cfg, void* d_ws, size_t ws_bytes, void* stream) {
    CallRange nvtx_range("px_partition");
    set_error("");
    px_status s = check_batch(in, "px_partition in");
    if (s != PX_OK) return s;
    s = check_batch(out, "px_partition out");
    if (s != PX_OK) return s;
    if (in->ncols < 1) return fail(PX_ERR_INVALID, "px_partition: input has no columns");
    if (key_col < 0 || key_col >= in->ncols) return fail(PX_ERR_INVALID, "px_partition: key_col %d", key_col);
    if (in->cols[key_col].type != PX_I64) return fail(PX_ERR_INVALID, "px_partition: key column must be PX_I64");
    if (nparts < 1 || nparts > PX_MAX_PARTS)
        return fail(PX_ERR_UNSUPPORTED, "px_partition: nparts %d outside [1, %d]", nparts, PX_MAX_PARTS);
    if ((d_sel == nullptr) != (d_nsel == nullptr))
        return fail(PX_ERR_INVALID, "px_partition: d_sel and d_nsel must be given together");
    if (out->ncols != in->ncols) return fail(PX_ERR_INVALID, "px_partition: out has %d columns, in has %d",
                                             out->ncols, in->ncols);
    for (int c = 0; c < in->ncols; ++c)
        if (out->cols[c].type != in->cols[c].type)
            return fail(PX_ERR_INVALID, "px_partition: column %d type differs between in and out", c);
    if (out->nrows < in->nrows)
        return fail(PX_ERR_INVALID, "px_partition: out capacity %lld below input rows %lld",
                    (long long)out->nrows, (long long)in->nrows);
    if (!d_offsets) return fail(PX_ERR_INVALID, "px_partition: null d_offsets");
    int32_t items_req = 0, bps = 0;
    if (cfg) {
        if (cfg->items != 0 && cfg->items != 2 && cfg->items != 4 && cfg->items != 8)
            return fail(PX_ERR_INVALID, "px_partition: config items %d (0, 2, 4 or 8)", cfg->items);
        if (cfg->blocks_per_sm < 0 || cfg->blocks_per_sm > 32)
            return fail(PX_ERR_INVALID, "px_partition: config blocks_per_sm %d (0..32)", cfg->blocks_per_sm);
        items_req = cfg->items;
        bps = cfg->blocks_per_sm;
    }
    const int64_t ncap = in->nrows;
    s = check_ws(d_ws, ws_bytes, px_partition_ws_bytes(ncap, nparts), "px_partition");
    if (s != PX_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (ncap == 0) {
        cudaMemsetAsync(d_offsets, 0, sizeof(int64_t) * (nparts + 1), st);
        return check_launch("px_partition");
    }
    Cols cols;
    cols.ncols = in->ncols;
    uint32_t row_bytes = 0;
    for (int c = 0; c < in->ncols; ++c) {
        cols.width[c] = in->cols[c].type;
        cols.in[c] = in->cols[c].data;
        cols.out[c] = out->cols[c].data;
        row_bytes += static_cast<uint32_t>(in->cols[c].type);
    }
    // Move order: decreasing width (stable), so each column's partition-ordered
    // buffer can be the staging area of the column moved before it.
    int n_ord = 0;
    for (int w : {8, 4, 1})
        for (int c = 0; c < in->ncols; ++c)
            if (cols.width[c] == w) cols.order[n_ord++] = c;
    // Rows per thread: the caller's choice when a tile of every column fits the
    // staging budget, else the widest that fits.
    const int fit = items_for(row_bytes);
    const int items = items_req > 0 && items_req <= fit ? items_req : fit;
    const int64_t T = static_cast<int64_t>(kThreads) * items;
    uint32_t stage_bytes = 0;
    for (int c = 0; c < in->ncols; ++c) {
        cols.stage_off[c] = stage_bytes;
        stage_bytes += static_cast<uint32_t>(align_up(static_cast<size_t>(T) * cols.width[c], 16));
    }
    const int64_t ntiles = cdiv(ncap, T);
    const PartScratch ps = part_scratch(d_ws, ncap, ntiles, nparts);
    int32_t* status = &static_cast<WsHeader*>(d_ws)->status;
    const int64_t* d_n = d_sel ? d_nsel : in->d_nrows;
    if (items == 8)
        return launch_partition<8>(cols, key_col, d_sel, d_n, ncap, seed, nparts, d_offsets, ps, ntiles, stage_bytes,
                                   row_bytes, bps, status, st);
    if (items == 4)
        return launch_partition<4>(cols, key_col, d_sel, d_n, ncap, seed, nparts, d_offsets, ps, ntiles, stage_bytes,
                                   row_bytes, bps, status, st);
    return launch_partition<2>(cols, key_col, d_sel, d_n, ncap, seed, nparts, d_offsets, ps, ntiles, stage_bytes,
                               row_bytes, bps, status, st);
}

px_status px_partition(const px_batch* in, int32_t key_col, const int32_t* d_sel, const int64_t* d_nsel,
                       int32_t nparts, uint64_t seed, const px_batch* out, int64_t* d_offsets, void* d_ws,
                       size_t ws_bytes, void* stream) {
    return px_partition_tuned(in, key_col, d_sel, d_nsel, nparts, seed, out, d_offsets, nullptr, d_ws, ws_bytes,
                              stream);
}

}  // extern "C"
