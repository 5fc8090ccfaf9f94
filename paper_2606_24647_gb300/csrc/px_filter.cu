// px_filter: FilterProject's predicate (Sec. 3.2) as one single-pass stream
// compaction. Each block takes the next tile in launch order, evaluates
// lo <= col < hi for its 2048 rows (8 rows per thread, warp-contiguous), counts the
// passing rows with warp ballots, gets the tile's output offset from a bounded
// decoupled look-back, and writes the passing row indices in ascending order.
// HBM traffic: the column once plus 4 bytes per passing row.
#include "px_common.cuh"

namespace px {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;
constexpr int kWarps = kThreads / 32;

template <typename T>
__global__ void __launch_bounds__(kThreads)
filter_kernel(const T* __restrict__ col, int64_t ncap, const int64_t* __restrict__ d_nrows,
              int64_t lo, int64_t hi, int32_t* __restrict__ sel, int64_t* __restrict__ d_nsel,
              ScanScratch scan, int32_t* status, int64_t ntiles) {
    __shared__ int64_t s_tile;
    __shared__ int64_t s_excl;
    __shared__ int32_t s_warp[kWarps];
    const int64_t tile = next_tile(scan.counter, &s_tile);
    const int64_t n = actual_rows(d_nrows, ncap);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = tile * kTile + warp * (32 * kItems);

    T v[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int64_t r = base + i * 32 + lane;
        v[i] = r < n ? col[r] : T(0);
    }
    uint32_t mask[kItems];
    int32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int64_t r = base + i * 32 + lane;
        const int64_t x = static_cast<int64_t>(v[i]);
        mask[i] = __ballot_sync(FULL, r < n && lo <= x && x < hi);
        cnt += __popc(mask[i]);
    }
    if (lane == 0) s_warp[warp] = cnt;
    __syncthreads();
    if (warp == 0) {
        const int32_t w = lane < kWarps ? s_warp[lane] : 0;
        const int32_t incl = warp_incl_scan(w);
        const int32_t total = __shfl_sync(FULL, incl, 31);
        if (lane < kWarps) s_warp[lane] = incl - w;
        const int64_t excl = lookback(scan.states, tile, total, status);
        if (lane == 0) {
            s_excl = excl;
            if (tile == ntiles - 1) *d_nsel = excl + total;
        }
    }
    __syncthreads();
    int64_t pos = s_excl + s_warp[warp];
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        if (mask[i] & (1u << lane))
            sel[pos + __popc(mask[i] & lt)] = static_cast<int32_t>(base + i * 32 + lane);
        pos += __popc(mask[i]);
    }
}

}  // namespace
}  // namespace px

using namespace px;

extern "C" {

size_t px_filter_ws_bytes(int64_t nrows) {
    if (nrows < 0) nrows = 0;
    return kWsScratch + scan_scratch_bytes(cdiv(nrows, kTile));
}

px_status px_filter(const px_col* col, int64_t nrows, const int64_t* d_nrows, int64_t lo, int64_t hi,
                    int32_t* d_sel, int64_t* d_nsel, void* d_ws, size_t ws_bytes, void* stream) {
    set_error("");
    px_status s = check_col(col, "px_filter col", nrows == 0);
    if (s != PX_OK) return s;
    if (nrows < 0 || nrows > INT32_MAX)
        return fail(PX_ERR_UNSUPPORTED, "px_filter: nrows %lld outside [0, 2^31)", (long long)nrows);
    if (!d_sel || !d_nsel) return fail(PX_ERR_INVALID, "px_filter: null d_sel or d_nsel");
    s = check_ws(d_ws, ws_bytes, px_filter_ws_bytes(nrows), "px_filter");
    if (s != PX_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (nrows == 0) {
        cudaMemsetAsync(d_nsel, 0, sizeof(int64_t), st);
        return check_launch("px_filter");
    }
    const int64_t ntiles = cdiv(nrows, kTile);
    char* scratch = static_cast<char*>(d_ws) + kWsScratch;
    cudaMemsetAsync(scratch, 0, scan_scratch_bytes(ntiles), st);
    const ScanScratch scan = scan_scratch(scratch);
    int32_t* status = &static_cast<WsHeader*>(d_ws)->status;
    const dim3 grid(static_cast<unsigned>(ntiles));
    switch (col->type) {
        case PX_I8:
            filter_kernel<int8_t><<<grid, kThreads, 0, st>>>(static_cast<const int8_t*>(col->data), nrows,
                                                             d_nrows, lo, hi, d_sel, d_nsel, scan, status, ntiles);
            break;
        case PX_I32:
            filter_kernel<int32_t><<<grid, kThreads, 0, st>>>(static_cast<const int32_t*>(col->data), nrows,
                                                              d_nrows, lo, hi, d_sel, d_nsel, scan, status, ntiles);
            break;
        default:
            filter_kernel<int64_t><<<grid, kThreads, 0, st>>>(static_cast<const int64_t*>(col->data), nrows,
                                                              d_nrows, lo, hi, d_sel, d_nsel, scan, status, ntiles);
            break;
    }
    note_launch();
    return check_launch("px_filter");
}

}  // extern "C"
