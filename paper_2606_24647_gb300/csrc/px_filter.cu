// px_filter: FilterProject's predicate (Sec. 3.2) as a stream compaction in three
// launches over tiles of 2048 rows (8 rows per thread, warp-contiguous):
//   1. count - per tile, the rows with lo <= col < hi (warp ballots) -> cnt[tile];
//   2. scan  - one block scans cnt in place into each tile's output start and
//              writes the total to *d_nsel;
//   3. write - per tile, the ballots again, a block scan of the warps' counts and
//              the tile's start give every passing row its slot in ascending order.
// Every tile is independent in launches 1 and 3. A single pass with a decoupled
// look-back measured 4-7x slower at 6M-60M rows: with about a thousand tiles in
// flight each tile walked back hundreds of predecessors to a published prefix.
// HBM traffic: the column twice (the second read hits L2 when the column fits)
// plus 4 bytes per passing row.
#include <mutex>

#include "px_common.cuh"

namespace px {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;
constexpr int kWarps = kThreads / 32;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;  // counts per thread per round of the scan

// Ballots of rows [base, base + 32 * kItems) of one warp (row base + 32 i + lane).
template <typename T>
__device__ __forceinline__ int32_t tile_masks(const T* __restrict__ col, int64_t base, int64_t n, int64_t lo,
                                              int64_t hi, int lane, uint32_t* mask) {
    T v[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int64_t r = base + i * 32 + lane;
        v[i] = r < n ? col[r] : T(0);
    }
    int32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int64_t r = base + i * 32 + lane;
        const int64_t x = static_cast<int64_t>(v[i]);
        mask[i] = __ballot_sync(FULL, r < n && lo <= x && x < hi);
        cnt += __popc(mask[i]);
    }
    return cnt;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
filter_count_kernel(const T* __restrict__ col, int64_t ncap, const int64_t* __restrict__ d_nrows, int64_t lo,
                    int64_t hi, int32_t* __restrict__ cnt) {
    __shared__ int32_t s_warp[kWarps];
    const int64_t n = actual_rows(d_nrows, ncap);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t mask[kItems];
    const int32_t c = tile_masks(col, static_cast<int64_t>(blockIdx.x) * kTile + warp * (32 * kItems), n, lo, hi,
                                 lane, mask);
    if (lane == 0) s_warp[warp] = c;
    __syncthreads();
    if (warp == 0) {
        const int32_t t = warp_sum(lane < kWarps ? s_warp[lane] : 0);
        if (lane == 0) cnt[blockIdx.x] = t;
    }
}

// One block: exclusive scan of cnt[0, ntiles) in place, rounds of
// kScanThreads * kScanItems counts (each thread a contiguous run), carried across
// rounds; *d_nsel = the total.
__global__ void __launch_bounds__(kScanThreads)
filter_scan_kernel(int32_t* __restrict__ cnt, int64_t ntiles, int64_t* __restrict__ d_nsel) {
    __shared__ int32_t s_warp[kScanThreads / 32];
    __shared__ int32_t s_total;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int32_t carry = 0;  // passing rows fit int32: nrows < 2^31
    for (int64_t r0 = 0; r0 < ntiles; r0 += kScanThreads * kScanItems) {
        const int64_t b = r0 + static_cast<int64_t>(tid) * kScanItems;
        int32_t v[kScanItems];
        int32_t sum = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            v[k] = b + k < ntiles ? cnt[b + k] : 0;
            sum += v[k];
        }
        const int32_t incl = warp_incl_scan(sum);
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int32_t w = s_warp[lane];
            const int32_t wi = warp_incl_scan(w);
            s_warp[lane] = wi - w;
            if (lane == 31) s_total = wi;
        }
        __syncthreads();
        int32_t run = carry + s_warp[warp] + incl - sum;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (b + k < ntiles) cnt[b + k] = run;
            run += v[k];
        }
        carry += s_total;
        __syncthreads();  // s_warp and s_total are rewritten by the next round
    }
    if (tid == 0) *d_nsel = carry;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
filter_write_kernel(const T* __restrict__ col, int64_t ncap, const int64_t* __restrict__ d_nrows, int64_t lo,
                    int64_t hi, const int32_t* __restrict__ start, int32_t* __restrict__ sel) {
    __shared__ int32_t s_warp[kWarps];
    const int64_t n = actual_rows(d_nrows, ncap);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile + warp * (32 * kItems);
    const int32_t tile_start = start[blockIdx.x];
    uint32_t mask[kItems];
    const int32_t c = tile_masks(col, base, n, lo, hi, lane, mask);
    if (lane == 0) s_warp[warp] = c;
    __syncthreads();
    if (warp == 0) {
        const int32_t w = lane < kWarps ? s_warp[lane] : 0;
        const int32_t incl = warp_incl_scan(w);
        if (lane < kWarps) s_warp[lane] = incl - w;
    }
    __syncthreads();
    int64_t pos = static_cast<int64_t>(tile_start) + s_warp[warp];
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        if (mask[i] & (1u << lane)) sel[pos + __popc(mask[i] & lt)] = static_cast<int32_t>(base + i * 32 + lane);
        pos += __popc(mask[i]);
    }
}

template <typename T>
void launch_filter(const void* col, int64_t nrows, const int64_t* d_nrows, int64_t lo, int64_t hi, int32_t* d_sel,
                   int64_t* d_nsel, int32_t* cnt, int64_t ntiles, cudaStream_t st) {
    const T* c = static_cast<const T*>(col);
    const unsigned grid = static_cast<unsigned>(ntiles);
    filter_count_kernel<T><<<grid, kThreads, 0, st>>>(c, nrows, d_nrows, lo, hi, cnt);
    filter_scan_kernel<<<1, kScanThreads, 0, st>>>(cnt, ntiles, d_nsel);
    filter_write_kernel<T><<<grid, kThreads, 0, st>>>(c, nrows, d_nrows, lo, hi, cnt, d_sel);
}

// cnt: ntiles int32 of device scratch.
void launch_filter_type(int32_t type, const void* col, int64_t nrows, const int64_t* d_nrows, int64_t lo, int64_t hi,
                        int32_t* d_sel, int64_t* d_nsel, int32_t* cnt, int64_t ntiles, cudaStream_t st) {
    switch (type) {
        case PX_I8: launch_filter<int8_t>(col, nrows, d_nrows, lo, hi, d_sel, d_nsel, cnt, ntiles, st); break;
        case PX_I32: launch_filter<int32_t>(col, nrows, d_nrows, lo, hi, d_sel, d_nsel, cnt, ntiles, st); break;
        default: launch_filter<int64_t>(col, nrows, d_nrows, lo, hi, d_sel, d_nsel, cnt, ntiles, st); break;
    }
    note_launch();
    note_launch();
    note_launch();
}

size_t count_bytes(int64_t ntiles) { return align_up(static_cast<size_t>(ntiles) * 4, 256); }

}  // namespace
}  // namespace px

using namespace px;

extern "C" {

size_t px_filter_ws_bytes(int64_t nrows) {
    if (nrows < 0) nrows = 0;
    return kWsScratch + count_bytes(cdiv(nrows, kTile));
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
    int32_t* cnt = reinterpret_cast<int32_t*>(static_cast<char*>(d_ws) + kWsScratch);
    launch_filter_type(col->type, col->data, nrows, d_nrows, lo, hi, d_sel, d_nsel, cnt, ntiles, st);
    return check_launch("px_filter");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// px_filter_noalloc: the same filter for callers that cannot allocate device
// memory, so cannot provide a workspace: e.g. code running under a host engine
// whose memory manager owns every device byte and forbids side allocations, or a
// serving loop that reserves all memory at start-up and must not call cudaMalloc
// (which can synchronise the device) on its hot path. Its scratch (one count per
// tile, after a header kept for the workspace layout the filter kernels share)
// lives in the file-scope device array below instead of a caller workspace.
namespace px {
namespace {

constexpr int64_t kNoallocMaxTiles = 65536;  // PX_FILTER_NOALLOC_MAX_ROWS / kTile
static_assert(PX_FILTER_NOALLOC_MAX_ROWS == kNoallocMaxTiles * kTile, "row limit must match the scratch size");
// Header (status word) + one count per tile: 256 + 262,144 = 262,400 bytes.
constexpr size_t kNoallocScratchBytes = kWsScratch + kNoallocMaxTiles * 4;
static_assert(kNoallocScratchBytes == 262400, "documented size of the static scratch");

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
    if (kWsScratch + static_cast<size_t>(ntiles) * 4 > kNoallocScratchBytes)
        return fail(PX_ERR_UNSUPPORTED, "px_filter_noalloc: %lld tiles exceed the static scratch", (long long)ntiles);
    // The array keeps whatever the previous call left there; every count a call
    // uses is written before it is read, so nothing needs clearing. The filter
    // records no data-dependent error, so the status is always PX_OK.
    if (nrows == 0) {
        cudaMemsetAsync(d_nsel, 0, sizeof(int64_t), st);
    } else {
        int32_t* cnt = reinterpret_cast<int32_t*>(static_cast<char*>(scratch) + kWsScratch);
        launch_filter_type(col->type, col->data, nrows, d_nrows, lo, hi, d_sel, d_nsel, cnt, ntiles, st);
    }
    if (d_status) cudaMemsetAsync(d_status, 0, sizeof(int32_t), st);
    return check_launch("px_filter_noalloc");
}
