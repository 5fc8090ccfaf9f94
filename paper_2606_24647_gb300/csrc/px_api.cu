// Host-side plumbing of the px C ABI: error reporting, argument checks, the
// workspace status word.
#include <atomic>
#include <string>

#include "px_common.cuh"

namespace px {

static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

px_status fail(px_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

px_status check_launch(const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PX_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return PX_OK;
}

px_status check_col(const px_col* c, const char* what, bool empty) {
    if (!c) return fail(PX_ERR_INVALID, "%s: null column descriptor", what);
    if (!valid_type(c->type)) return fail(PX_ERR_INVALID, "%s: unknown column type %d", what, c->type);
    if (c->reserved != 0) return fail(PX_ERR_INVALID, "%s: reserved field must be 0", what);
    if (!c->data && !empty) return fail(PX_ERR_INVALID, "%s: null column data", what);
    if (!aligned16(c->data)) return fail(PX_ERR_INVALID, "%s: column data not 16-byte aligned", what);
    return PX_OK;
}

px_status check_batch(const px_batch* b, const char* what) {
    if (!b) return fail(PX_ERR_INVALID, "%s: null batch", what);
    if (b->ncols < 0 || b->ncols > PX_MAX_COLS)
        return fail(PX_ERR_UNSUPPORTED, "%s: %d columns (1..%d supported)", what, b->ncols, PX_MAX_COLS);
    if (b->ncols > 0 && !b->cols) return fail(PX_ERR_INVALID, "%s: null column array", what);
    if (b->reserved != 0) return fail(PX_ERR_INVALID, "%s: reserved field must be 0", what);
    if (b->nrows < 0 || b->nrows > INT32_MAX)
        return fail(PX_ERR_UNSUPPORTED, "%s: nrows %lld outside [0, 2^31)", what, (long long)b->nrows);
    for (int i = 0; i < b->ncols; ++i) {
        char w[96];
        snprintf(w, sizeof(w), "%s column %d", what, i);
        const px_status s = check_col(&b->cols[i], w, b->nrows == 0);
        if (s != PX_OK) return s;
    }
    return PX_OK;
}

px_status check_ws(const void* d_ws, size_t ws_bytes, size_t need, const char* what) {
    if (!d_ws) return fail(PX_ERR_INVALID, "%s: null workspace", what);
    if (!aligned16(d_ws)) return fail(PX_ERR_INVALID, "%s: workspace not 16-byte aligned", what);
    if (ws_bytes < need)
        return fail(PX_ERR_INVALID, "%s: workspace of %zu bytes, %zu needed", what, ws_bytes, need);
    return PX_OK;
}

}  // namespace px

using namespace px;

extern "C" {

const char* px_last_error(void) { return g_last_error.c_str(); }

uint64_t px_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

px_status px_ws_init(void* d_ws, size_t ws_bytes, void* stream) {
    g_last_error.clear();
    const px_status s = check_ws(d_ws, ws_bytes, kWsHeader, "px_ws_init");
    if (s != PX_OK) return s;
    if (cudaMemsetAsync(d_ws, 0, kWsHeader, static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return check_launch("px_ws_init memset");
    return PX_OK;
}

px_status px_stream_status(void* stream, const void* d_ws) {
    g_last_error.clear();
    if (!d_ws) return fail(PX_ERR_INVALID, "px_stream_status: null workspace");
    int32_t st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, d_ws, sizeof(st), cudaMemcpyDeviceToHost,
                                    static_cast<cudaStream_t>(stream));
    if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(PX_ERR_CUDA, "px_stream_status: %s", cudaGetErrorString(e));
    if (st != PX_OK) set_error("device status %d recorded in workspace", st);
    return st;
}

}  // extern "C"

namespace px {
namespace {

__global__ void selftest_wait_kernel(const int32_t* flag, uint32_t limit, int32_t* status) {
    for (uint32_t i = 0; i < limit; ++i) {
        int32_t v;
        asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v != 0) {
            *status = PX_OK;
            return;
        }
        __nanosleep(64);
    }
    *status = PX_ERR_TIMEOUT;
}

}  // namespace
}  // namespace px

extern "C" px_status px_selftest_wait(const int32_t* d_flag, uint32_t spin_limit, int32_t* d_status, void* stream) {
    using namespace px;
    set_error("");
    if (!d_flag || !d_status) return fail(PX_ERR_INVALID, "px_selftest_wait: null pointer");
    if (spin_limit < 1 || spin_limit > (1u << 24))
        return fail(PX_ERR_INVALID, "px_selftest_wait: spin_limit %u outside [1, 2^24]", spin_limit);
    selftest_wait_kernel<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(d_flag, spin_limit, d_status);
    note_launch();
    return check_launch("px_selftest_wait");
}
