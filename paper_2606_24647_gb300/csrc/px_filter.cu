// px_filter: FilterProject's predicate (Sec. 3.2) as one single-pass stream
// compaction. Each block takes the next tile in launch order, evaluates
// lo <= col < hi for its 2048 rows (8 rows per thread, warp-contiguous), counts the
// passing rows with warp ballots, gets the tile's output offset from a bounded
// decoupled look-back, and writes the passing row indices in ascending order.
// HBM traffic: the column once plus 4 bytes per passing row.
#include <mutex>

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
    CallRange nvtx_range("px_filter");
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

// ---------------------------------------------------------------------------
// px_filter_noalloc: the same filter for callers that cannot allocate device
// memory, so cannot provide a workspace: e.g. code running under a host engine
// whose memory manager owns every device byte and forbids side allocations, or a
// serving loop that reserves all memory at start-up and must not call cudaMalloc
// (which can synchronise the device) on its hot path. Its scratch (the status
// word, the tile counter and one look-back state per tile) lives in the
// file-scope device array below instead of a caller workspace.
namespace px {
namespace {

constexpr int64_t kNoallocMaxTiles = 65536;  // PX_FILTER_NOALLOC_MAX_ROWS / kTile
static_assert(PX_FILTER_NOALLOC_MAX_ROWS == kNoallocMaxTiles * kTile, "row limit must match the scratch size");
// Header (status word) + scan scratch for the largest tile count, rounded like
// scan_scratch_bytes: 256 + 524,544 = 524,800 bytes.
constexpr size_t kNoallocScratchBytes = kWsScratch + ((16 + 8 * kNoallocMaxTiles + 255) / 256) * 256;

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_filter_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of g_filter_scratch on the current device. In host code the
// array's name is only a host-side stand-in, so the address is looked up once per
// device with cudaGetSymbolAddress (with that device current) and cached.
px_status noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PX_ERR_CUDA, "px_filter_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(PX_ERR_UNSUPPORTED, "px_filter_noalloc: device %d", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_filter_scratch);
        if (e != cudaSuccess || !p)
            return fail(PX_ERR_CUDA, "px_filter_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return PX_OK;
}

}  // namespace
}  // namespace px

extern "C" px_status px_filter_noalloc(const px_col* col, int64_t nrows, const int64_t* d_nrows, int64_t lo,
                                       int64_t hi, int32_t* d_sel, int64_t* d_nsel, int32_t* d_status,
                                       void* stream) {
    CallRange nvtx_range("px_filter_noalloc");
    set_error("");
    px_status s = check_col(col, "px_filter_noalloc col", nrows == 0);
    if (s != PX_OK) return s;
    if (nrows < 0 || nrows > PX_FILTER_NOALLOC_MAX_ROWS)
        return fail(PX_ERR_UNSUPPORTED, "px_filter_noalloc: nrows %lld outside [0, %lld]; use px_filter",
                    (long long)nrows, (long long)PX_FILTER_NOALLOC_MAX_ROWS);
    if (!d_sel || !d_nsel) return fail(PX_ERR_INVALID, "px_filter_noalloc: null d_sel or d_nsel");
    void* scratch = nullptr;
    if ((s = noalloc_scratch(&scratch)) != PX_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t ntiles = cdiv(nrows, kTile);
    if (kWsScratch + scan_scratch_bytes(ntiles) > kNoallocScratchBytes)
        return fail(PX_ERR_UNSUPPORTED, "px_filter_noalloc: %lld tiles exceed the static scratch", (long long)ntiles);
    // Each call clears the status word, the tile counter and the states it uses:
    // the array keeps whatever the previous call left there.
    cudaMemsetAsync(scratch, 0, kWsScratch + scan_scratch_bytes(ntiles), st);
    if (nrows == 0) {
        cudaMemsetAsync(d_nsel, 0, sizeof(int64_t), st);
    } else {
        const ScanScratch scan = scan_scratch(static_cast<char*>(scratch) + kWsScratch);
        int32_t* status = &static_cast<WsHeader*>(scratch)->status;
        const dim3 grid(static_cast<unsigned>(ntiles));
        switch (col->type) {
            case PX_I8:
                filter_kernel<int8_t><<<grid, kThreads, 0, st>>>(static_cast<const int8_t*>(col->data), nrows,
                                                                 d_nrows, lo, hi, d_sel, d_nsel, scan, status, ntiles);
                break;
            case PX_I32:
                filter_kernel<int32_t><<<grid, kThreads, 0, st>>>(static_cast<const int32_t*>(col->data), nrows,
                                                                  d_nrows, lo, hi, d_sel, d_nsel, scan, status,
                                                                  ntiles);
                break;
            default:
                filter_kernel<int64_t><<<grid, kThreads, 0, st>>>(static_cast<const int64_t*>(col->data), nrows,
                                                                  d_nrows, lo, hi, d_sel, d_nsel, scan, status,
                                                                  ntiles);
                break;
        }
        note_launch();
    }
    if (d_status) cudaMemcpyAsync(d_status, scratch, sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    return check_launch("px_filter_noalloc");
}
