// Shared device and host helpers of the px CUDA library (sm_103a).
//
// Everything here is the CUDA path's own code; none of it is shared with the CPU
// oracle. The hash is written from the published definition of MurmurHash3's
// 64-bit finalizer; the single-pass prefix scan is the decoupled look-back scan
// of Merrill & Garland ("Single-pass Parallel Prefix Scan with Decoupled
// Look-back", 2016) with every wait bounded.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>

#include <nvtx3/nvToolsExt.h>

#include "px.h"

namespace px {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------- workspace --
// d_ws layout: [0, 256) header; scratch of each call from kWsScratch on.
constexpr size_t kWsHeader = 256;
constexpr size_t kWsScratch = kWsHeader;

struct WsHeader {
    int32_t status;     // sticky: first data-dependent error wins
    int32_t reserved;
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Scratch of a single-pass scan over `ntiles` tiles: a dynamic tile counter and one
// 64-bit state word per tile, zeroed before each launch.
inline size_t scan_scratch_bytes(int64_t ntiles) { return align_up(16 + 8 * (size_t)ntiles, 256); }

// ------------------------------------------------------------ device status --
__device__ __forceinline__ void set_status(int32_t* st, int32_t code) { atomicCAS(st, 0, code); }

// Bound of every device-side spin wait: about a second of polling, after which the
// waiter records PX_ERR_TIMEOUT and carries on without the awaited value.
constexpr uint32_t kSpinLimit = 1u << 21;

// --------------------------------------------------------------------- hash --
// MurmurHash3 64-bit finalizer: xor-shift 33, multiply, xor-shift 33, multiply,
// xor-shift 33 (constants from the published MurmurHash3 source).
__device__ __forceinline__ uint64_t fmix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

// Partition of a key: upper 32 hash bits reduced to [0, nparts) by multiply-shift.
__device__ __forceinline__ uint32_t part_of(int64_t key, uint64_t seed, uint32_t nparts) {
    const uint64_t h = fmix64(static_cast<uint64_t>(key) ^ seed);
    return __umulhi(static_cast<uint32_t>(h >> 32), nparts);
}

// Slot of a key in a table segment of `cap` slots: the LOWER 32 hash bits reduced
// by multiply-shift, so slot choice is independent of the partition bits.
__device__ __forceinline__ uint32_t slot_of(uint64_t h, uint32_t cap) {
    return __umulhi(static_cast<uint32_t>(h), cap);
}

// ------------------------------------------------------------ typed columns --
__device__ __forceinline__ int64_t load_int(const void* p, int w, int64_t i) {
    if (w == 8) return static_cast<const int64_t*>(p)[i];
    if (w == 4) return static_cast<int64_t>(static_cast<const int32_t*>(p)[i]);
    return static_cast<int64_t>(static_cast<const int8_t*>(p)[i]);
}

__device__ __forceinline__ void store_int(void* p, int w, int64_t i, int64_t v) {
    if (w == 8) static_cast<int64_t*>(p)[i] = v;
    else if (w == 4) static_cast<int32_t*>(p)[i] = static_cast<int32_t>(v);
    else static_cast<int8_t*>(p)[i] = static_cast<int8_t>(v);
}

// --------------------------------------------------------------- warp utils --
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T u = __shfl_up_sync(FULL, v, d);
        if (lane >= d) v += u;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
    return v;
}

// Sum mod 2^64 of x over the 32 lanes of a warp (all lanes call it): three 32-bit
// warp reductions (redux.sync) - the low word as two 16-bit halves, whose sums
// cannot overflow, and the high word mod 2^32 - instead of a 64-bit shuffle
// butterfly (five rounds of two shuffles and a 64-bit add).
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t x) {
    const uint32_t lo = static_cast<uint32_t>(x), hi = static_cast<uint32_t>(x >> 32);
    const uint32_t s0 = __reduce_add_sync(FULL, lo & 0xffffu);
    const uint32_t s1 = __reduce_add_sync(FULL, lo >> 16);
    const uint32_t sh = __reduce_add_sync(FULL, hi);
    return static_cast<uint64_t>(s0) + (static_cast<uint64_t>(s1) << 16) + (static_cast<uint64_t>(sh) << 32);
}

// In-place exclusive scan of s[0..n) in shared memory by the whole block
// (n <= 4 * blockDim.x, blockDim.x a multiple of 32, <= 1024). `s_warp` holds 33
// ints. Returns the total. Contains __syncthreads: call from all threads.
__device__ __forceinline__ int32_t block_excl_scan_smem(int32_t* s, int n, int32_t* s_warp) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    int32_t v[4];
    int32_t sum = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int idx = tid * 4 + k;
        v[k] = idx < n ? s[idx] : 0;
        sum += v[k];
    }
    const int32_t incl = warp_incl_scan(sum);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int32_t w = lane < nwarps ? s_warp[lane] : 0;
        const int32_t wi = warp_incl_scan(w);
        if (lane < nwarps) s_warp[lane] = wi - w;
        if (lane == 31) s_warp[32] = wi;  // block total
    }
    __syncthreads();
    int32_t run = s_warp[warp] + incl - sum;
    const int32_t total = s_warp[32];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int idx = tid * 4 + k;
        if (idx < n) s[idx] = run;
        run += v[k];
    }
    __syncthreads();
    return total;
}

// ---------------------------------------------------- decoupled look-back ----
constexpr uint64_t kLbAgg = 1ull << 62;   // tile aggregate published
constexpr uint64_t kLbPre = 2ull << 62;   // tile inclusive prefix published
constexpr uint64_t kLbVal = (1ull << 62) - 1;

__device__ __forceinline__ uint64_t ld_acquire(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint64_t* p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

struct ScanScratch {
    unsigned long long* counter;  // dynamic tile ids
    uint64_t* states;             // one word per tile
};

__host__ __device__ inline ScanScratch scan_scratch(void* base) {
    ScanScratch s;
    s.counter = static_cast<unsigned long long*>(base);
    s.states = reinterpret_cast<uint64_t*>(static_cast<char*>(base) + 16);
    return s;
}

// Tile id in launch order, so a tile only ever waits on tiles whose blocks are
// already running. Call from all threads; contains __syncthreads.
__device__ __forceinline__ int64_t next_tile(unsigned long long* counter, int64_t* s_slot) {
    if (threadIdx.x == 0) *s_slot = static_cast<int64_t>(atomicAdd(counter, 1ull));
    __syncthreads();
    return *s_slot;
}

// Exclusive prefix of `tile` given its aggregate. Called by all 32 lanes of ONE
// warp; every lane gets the result. Publishes the tile's inclusive prefix.
__device__ __forceinline__ int64_t lookback(uint64_t* states, int64_t tile, int64_t aggregate,
                                            int32_t* status) {
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) st_release(&states[0], kLbPre | static_cast<uint64_t>(aggregate));
        return 0;
    }
    if (lane == 0) st_release(&states[tile], kLbAgg | static_cast<uint64_t>(aggregate));
    int64_t excl = 0;
    int64_t base = tile - 1;
    uint32_t spins = 0;
    while (true) {
        const int64_t idx = base - lane;
        const uint64_t s = idx >= 0 ? ld_acquire(&states[idx]) : kLbPre;
        const uint32_t flag = static_cast<uint32_t>(s >> 62);
        if (__any_sync(FULL, flag == 0)) {
            if (++spins > kSpinLimit) {
                if (lane == 0) set_status(status, PX_ERR_TIMEOUT);
                break;
            }
            __nanosleep(100);
            continue;
        }
        const uint32_t pre = __ballot_sync(FULL, flag == 2);
        int64_t v = static_cast<int64_t>(s & kLbVal);
        if (pre) {
            if (lane > __ffs(pre) - 1) v = 0;
            excl += warp_sum(v);
            break;
        }
        excl += warp_sum(v);
        base -= 32;
    }
    if (lane == 0) st_release(&states[tile], kLbPre | static_cast<uint64_t>(excl + aggregate));
    return excl;
}

// ------------------------------------------------- TMA bulk copies (sm_90+) --
// One-dimensional bulk copies global -> shared completed on an mbarrier
// (cp.async.bulk ... mbarrier::complete_tx). Source and destination must be
// 16-byte aligned and the size a multiple of 16 bytes.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Makes the initialised barrier visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the barrier's phase `parity` to complete: false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ------------------------------------------- programmatic dependent launch --
// A kernel launched with launch_after() may start while the kernel before it on the
// stream is still running (once every block of that one has called
// allow_dependents() or exited); it must call wait_prior() before it reads anything
// that kernel writes. Work that needs no such data (staging inputs of earlier
// calls, clearing shared memory) runs before the wait and overlaps the tail of the
// kernel before. wait_prior() returns when the kernel before has completed and its
// memory is visible; since that kernel waited for its own predecessor the same way,
// the whole stream before is then complete.
__device__ __forceinline__ void wait_prior() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" :::); }

template <typename... Params, typename... Args>
cudaError_t launch_after(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                         Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Params>(args)...);
}

// ------------------------------------------------------------ reductions --
// Fire-and-forget reductions (PTX red): no old value comes back, so the issuing
// warp never waits on the memory system for them.
__device__ __forceinline__ void red_add_global(unsigned long long* p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "l"(v) : "memory");
}
__device__ __forceinline__ void red_add_shared(uint32_t* p, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void red_or_shared(uint32_t* p, uint32_t v) {
    asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}

// Row count of a batch or selection: the device count when given (clamped to the
// capacity), else the host count.
__device__ __forceinline__ int64_t actual_rows(const int64_t* d_n, int64_t cap) {
    if (!d_n) return cap;
    const int64_t n = *d_n;
    return n < 0 ? 0 : (n < cap ? n : cap);
}

__device__ __forceinline__ int seg_of(const int64_t* seg, int nsegs, int64_t pos) {
    // largest q in [0, nsegs) with seg[q] <= pos
    int lo = 0, hi = nsegs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg[mid] <= pos) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// --------------------------------------------------------------------- host --
void set_error(const char* fmt, ...);
px_status fail(px_status code, const char* fmt, ...);
px_status check_launch(const char* what);
void note_launch();  // counts one kernel launch (px_kernel_launches)

// NVTX range around one C-ABI call (host enqueue time), named after the call, for
// timeline tools; free when no tool is attached.
struct CallRange {
    explicit CallRange(const char* name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
    CallRange(const CallRange&) = delete;
    CallRange& operator=(const CallRange&) = delete;
};

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline bool valid_type(int32_t t) { return t == PX_I8 || t == PX_I32 || t == PX_I64; }

// A column's data may be null only when it has no rows (`empty`).
px_status check_col(const px_col* c, const char* what, bool empty);
px_status check_batch(const px_batch* b, const char* what);
px_status check_ws(const void* d_ws, size_t ws_bytes, size_t need, const char* what);

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Streaming multiprocessors of the current device.
inline int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace px
