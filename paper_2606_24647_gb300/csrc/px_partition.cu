// px_partition: PartitionedOutput's hash partitioning (Sec. 3.1, Sec. 3.3.2) as an
// on-device exchange. The output is one packed buffer per column holding partition
// 0's rows, then partition 1's, ... (stable), plus offsets[nparts+1]: the
// UcxExchange's "size metadata, then packed GPU data" for every destination.
//
// Three launches over tiles of 4096 positions:
//   1. hist    - per-tile partition counts, stored partition-major: cnt[q][t].
//   2. scan    - exclusive scan of cnt in that order gives each (partition, tile)
//                its global output start (single pass, bounded look-back), and
//                offsets[q] = start of (q, tile 0).
//   3. scatter - recomputes each row's partition, ranks rows stably inside the
//                tile (warp match_any + per-warp counters, rows in order), then
//                for each column stages the tile in shared memory grouped by
//                partition and writes each partition's run contiguously, so the
//                stores coalesce. The key column is read twice (hist and
//                scatter); every other column once; every column written once.
#include "px_common.cuh"

namespace px {
namespace {

constexpr int kThreads = 512;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;  // 4096 positions
constexpr int kWarps = kThreads / 32;

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

struct Cols {
    int32_t ncols;
    int32_t width[PX_MAX_COLS];
    const void* in[PX_MAX_COLS];
    void* out[PX_MAX_COLS];
};

// Local position of item i of this thread inside a tile: warp-contiguous runs of
// 32 * kItems positions, lanes innermost, so position order = (warp, item, lane).
__device__ __forceinline__ int local_pos(int warp, int i, int lane) { return warp * (32 * kItems) + i * 32 + lane; }

__global__ void __launch_bounds__(kThreads)
part_hist_kernel(const int64_t* __restrict__ key, const int32_t* __restrict__ sel,
                 const int64_t* __restrict__ d_nsel, int64_t ncap, uint64_t seed, uint32_t nparts,
                 int32_t* __restrict__ cnt, int64_t ntiles) {
    extern __shared__ int32_t s_hist[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (uint32_t q = tid; q < nparts; q += kThreads) s_hist[q] = 0;
    const int64_t n = actual_rows(d_nsel, ncap);
    const int64_t tbase = static_cast<int64_t>(blockIdx.x) * kTile;
    uint32_t p[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int64_t j = tbase + local_pos(warp, i, lane);
        p[i] = nparts;
        if (j < n) {
            const int64_t r = sel ? static_cast<int64_t>(sel[j]) : j;
            p[i] = part_of(key[r], seed, nparts);
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const uint32_t peers = __match_any_sync(FULL, p[i]);
        if (p[i] < nparts && lane == __ffs(peers) - 1) atomicAdd(&s_hist[p[i]], __popc(peers));
    }
    __syncthreads();
    for (uint32_t q = tid; q < nparts; q += kThreads) cnt[static_cast<int64_t>(q) * ntiles + blockIdx.x] = s_hist[q];
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
    const int64_t tile = next_tile(scan.counter, &s_tile);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = tile * kScanTile + static_cast<int64_t>(tid) * kScanItems;
    int32_t v[kScanItems];
    int32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < total ? cnt[base + k] : 0;
        sum += v[k];
    }
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
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t e = base + k;
        if (e < total) {
            offs[e] = static_cast<int32_t>(run);
            if (e % ntiles == 0) d_offsets[e / ntiles] = run;
        }
        run += v[k];
    }
}

template <typename T>
__device__ __forceinline__ void scatter_column(const Cols& cols, int c, bool is_key, const int64_t* keyv,
                                               const int32_t* rowv, const uint32_t* pidv, const int32_t* posv,
                                               uint32_t nparts, void* s_stage_raw, const uint16_t* s_pid,
                                               const int32_t* s_delta, int tile_rows) {
    T* s_stage = static_cast<T*>(s_stage_raw);
    const T* in = static_cast<const T*>(cols.in[c]);
    T val[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i)
        if (pidv[i] < nparts) val[i] = is_key ? static_cast<T>(keyv[i]) : in[rowv[i]];
#pragma unroll
    for (int i = 0; i < kItems; ++i)
        if (pidv[i] < nparts) s_stage[posv[i]] = val[i];
    __syncthreads();
    T* out = static_cast<T*>(cols.out[c]);
    for (int j = threadIdx.x; j < tile_rows; j += kThreads)
        out[static_cast<int64_t>(s_delta[s_pid[j]]) + j] = s_stage[j];
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads)
part_scatter_kernel(Cols cols, int32_t key_col, const int32_t* __restrict__ sel,
                    const int64_t* __restrict__ d_nsel, int64_t ncap, uint64_t seed, uint32_t nparts,
                    const int32_t* __restrict__ offs, int64_t ntiles) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int np1 = static_cast<int>(nparts) + 1;
    int64_t* s_stage = reinterpret_cast<int64_t*>(smem);                       // kTile x 8 B
    uint16_t* s_pid = reinterpret_cast<uint16_t*>(smem + kTile * 8);            // kTile
    int32_t* s_warp = reinterpret_cast<int32_t*>(smem + kTile * 10);            // 33 (+3 pad)
    int32_t* s_tstart = s_warp + 36;                                            // np1 (+pad)
    int32_t* s_delta = s_tstart + ((np1 + 3) & ~3);                              // nparts (+pad)
    int32_t* s_whist = s_delta + ((np1 + 3) & ~3);                               // kWarps x np1

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t tile = blockIdx.x;
    const int64_t n = actual_rows(d_nsel, ncap);
    const int64_t tbase = tile * kTile;
    const int64_t rem = n - tbase;
    const int tile_rows = rem <= 0 ? 0 : (rem < kTile ? static_cast<int>(rem) : kTile);
    for (int k = tid; k < kWarps * np1; k += kThreads) s_whist[k] = 0;

    const int64_t* key = static_cast<const int64_t*>(cols.in[key_col]);
    int64_t keyv[kItems];
    int32_t rowv[kItems];
    uint32_t pidv[kItems];
    int32_t posv[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int lp = local_pos(warp, i, lane);
        pidv[i] = nparts;
        rowv[i] = 0;
        keyv[i] = 0;
        if (lp < tile_rows) {
            const int64_t j = tbase + lp;
            rowv[i] = sel ? sel[j] : static_cast<int32_t>(j);
            keyv[i] = key[rowv[i]];
        }
    }
#pragma unroll
    for (int i = 0; i < kItems; ++i)
        if (local_pos(warp, i, lane) < tile_rows) pidv[i] = part_of(keyv[i], seed, nparts);
    __syncthreads();

    // Stable rank inside the warp's run: rows of the same partition earlier in
    // (item, lane) order, counted with match_any and a per-warp counter row.
    int32_t* wh = s_whist + warp * np1;
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const uint32_t p = pidv[i];
        const uint32_t peers = __match_any_sync(FULL, p);
        const int32_t b = wh[p];
        __syncwarp();
        if (lane == __ffs(peers) - 1) wh[p] = b + __popc(peers);
        __syncwarp();
        posv[i] = b + __popc(peers & lt);
    }
    __syncthreads();
    // Per partition: exclusive scan over warps (in place) and the tile's count.
    for (int q = tid; q < static_cast<int>(nparts); q += kThreads) {
        int32_t run = 0;
        for (int w = 0; w < kWarps; ++w) {
            const int32_t c = s_whist[w * np1 + q];
            s_whist[w * np1 + q] = run;
            run += c;
        }
        s_tstart[q] = run;
    }
    __syncthreads();
    block_excl_scan_smem(s_tstart, static_cast<int>(nparts), s_warp);
    for (int q = tid; q < static_cast<int>(nparts); q += kThreads)
        s_delta[q] = offs[static_cast<int64_t>(q) * ntiles + tile] - s_tstart[q];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        if (pidv[i] < nparts) {
            posv[i] += s_tstart[pidv[i]] + wh[pidv[i]];
            s_pid[posv[i]] = static_cast<uint16_t>(pidv[i]);
        }
    }
    __syncthreads();

    for (int c = 0; c < cols.ncols; ++c) {
        const bool is_key = (c == key_col);
        switch (cols.width[c]) {
            case 8:
                scatter_column<int64_t>(cols, c, is_key, keyv, rowv, pidv, posv, nparts, s_stage, s_pid, s_delta,
                                        tile_rows);
                break;
            case 4:
                scatter_column<int32_t>(cols, c, is_key, keyv, rowv, pidv, posv, nparts, s_stage, s_pid, s_delta,
                                        tile_rows);
                break;
            default:
                scatter_column<int8_t>(cols, c, is_key, keyv, rowv, pidv, posv, nparts, s_stage, s_pid, s_delta,
                                       tile_rows);
                break;
        }
    }
}

size_t scatter_smem_bytes(int32_t nparts) {
    const size_t np1 = static_cast<size_t>(nparts) + 1;
    const size_t np1p = (np1 + 3) & ~static_cast<size_t>(3);
    return kTile * 10 + 36 * 4 + np1p * 4 * 2 + kWarps * np1 * 4;
}

struct PartScratch {
    int32_t* cnt;
    int32_t* offs;
    void* scan;
    size_t scan_bytes;
};

PartScratch part_scratch(void* d_ws, int64_t ntiles, int32_t nparts) {
    PartScratch p;
    char* base = static_cast<char*>(d_ws) + kWsScratch;
    const size_t mat = align_up(static_cast<size_t>(ntiles) * nparts * 4, 256);
    p.cnt = reinterpret_cast<int32_t*>(base);
    p.offs = reinterpret_cast<int32_t*>(base + mat);
    p.scan = base + 2 * mat;
    p.scan_bytes = scan_scratch_bytes(cdiv(ntiles * nparts, kScanTile));
    return p;
}

}  // namespace
}  // namespace px

using namespace px;

extern "C" {

size_t px_partition_ws_bytes(int64_t nrows, int32_t nparts) {
    if (nrows < 0) nrows = 0;
    if (nparts < 1) nparts = 1;
    const int64_t ntiles = cdiv(nrows, kTile);
    const size_t mat = align_up(static_cast<size_t>(ntiles) * nparts * 4, 256);
    return kWsScratch + 2 * mat + scan_scratch_bytes(cdiv(ntiles * nparts, kScanTile));
}

px_status px_partition(const px_batch* in, int32_t key_col, const int32_t* d_sel, const int64_t* d_nsel,
                       int32_t nparts, uint64_t seed, const px_batch* out, int64_t* d_offsets, void* d_ws,
                       size_t ws_bytes, void* stream) {
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
    const int64_t ncap = in->nrows;
    s = check_ws(d_ws, ws_bytes, px_partition_ws_bytes(ncap, nparts), "px_partition");
    if (s != PX_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (ncap == 0) {
        cudaMemsetAsync(d_offsets, 0, sizeof(int64_t) * (nparts + 1), st);
        return check_launch("px_partition");
    }
    const int64_t ntiles = cdiv(ncap, kTile);
    const PartScratch ps = part_scratch(d_ws, ntiles, nparts);
    int32_t* status = &static_cast<WsHeader*>(d_ws)->status;
    const int64_t* d_n = d_sel ? d_nsel : in->d_nrows;
    const int64_t* key = static_cast<const int64_t*>(in->cols[key_col].data);

    part_hist_kernel<<<static_cast<unsigned>(ntiles), kThreads, nparts * sizeof(int32_t), st>>>(
        key, d_sel, d_n, ncap, seed, static_cast<uint32_t>(nparts), ps.cnt, ntiles);
    note_launch();
    if ((s = check_launch("px_partition hist")) != PX_OK) return s;

    const int64_t total = ntiles * nparts;
    const int64_t nscan = cdiv(total, kScanTile);
    cudaMemsetAsync(ps.scan, 0, ps.scan_bytes, st);
    part_scan_kernel<<<static_cast<unsigned>(nscan), kScanThreads, 0, st>>>(
        ps.cnt, ps.offs, total, ntiles, static_cast<uint32_t>(nparts), d_offsets, scan_scratch(ps.scan), status,
        nscan);
    note_launch();
    if ((s = check_launch("px_partition scan")) != PX_OK) return s;

    Cols cols;
    cols.ncols = in->ncols;
    for (int c = 0; c < in->ncols; ++c) {
        cols.width[c] = in->cols[c].type;
        cols.in[c] = in->cols[c].data;
        cols.out[c] = out->cols[c].data;
    }
    const size_t smem = scatter_smem_bytes(nparts);
    cudaFuncSetAttribute(part_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(scatter_smem_bytes(PX_MAX_PARTS)));
    part_scatter_kernel<<<static_cast<unsigned>(ntiles), kThreads, smem, st>>>(
        cols, key_col, d_sel, d_n, ncap, seed, static_cast<uint32_t>(nparts), ps.offs, ntiles);
    note_launch();
    return check_launch("px_partition scatter");
}

}  // extern "C"
