// px_gather: payload columns fetched by row id - the second half of late
// materialization (Sec. 2.3): the exchange and the join move only (key, row id),
// and the columns the aggregation needs are gathered for the surviving rows.
#include <algorithm>

#include "px_common.cuh"

namespace px {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 4;

struct GatherCols {
    int32_t ncols;
    int32_t width[PX_MAX_COLS];
    const void* in[PX_MAX_COLS];
    void* out[PX_MAX_COLS];
};

template <typename T>
__device__ __forceinline__ void gather_col(const void* in, void* out, const int32_t* idx, const int64_t* pos,
                                           const bool* ok) {
    T v[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i)
        if (ok[i]) v[i] = static_cast<const T*>(in)[idx[i]];
#pragma unroll
    for (int i = 0; i < kItems; ++i)
        if (ok[i]) static_cast<T*>(out)[pos[i]] = v[i];
}

// Grid-stride over tiles of kThreads x kItems positions; per tile every column is
// gathered with all of its loads issued before its stores.
__global__ void __launch_bounds__(kThreads)
gather_kernel(GatherCols c, const int32_t* __restrict__ idx, const int64_t* __restrict__ d_n, int64_t ncap,
              int64_t in_rows, int32_t* status) {
    const int64_t n = actual_rows(d_n, ncap);
    const int64_t ntiles = cdiv(n, static_cast<int64_t>(kThreads) * kItems);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int32_t r[kItems];
        int64_t pos[kItems];
        bool ok[kItems];
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            pos[i] = tile * (kThreads * kItems) + i * kThreads + threadIdx.x;
            r[i] = pos[i] < n ? idx[pos[i]] : -1;
            ok[i] = r[i] >= 0 && r[i] < in_rows;
            if (pos[i] < n && !ok[i]) set_status(status, PX_ERR_INVALID);
        }
        for (int k = 0; k < c.ncols; ++k) {
            if (c.width[k] == 8) gather_col<int64_t>(c.in[k], c.out[k], r, pos, ok);
            else if (c.width[k] == 4) gather_col<int32_t>(c.in[k], c.out[k], r, pos, ok);
            else gather_col<int8_t>(c.in[k], c.out[k], r, pos, ok);
        }
    }
}

}  // namespace
}  // namespace px

using namespace px;

extern "C" px_status px_gather(const px_batch* in, const int32_t* d_idx, const int64_t* d_n, const px_batch* out,
                               void* d_ws, size_t ws_bytes, void* stream) {
    CallRange nvtx_range("px_gather");
    set_error("");
    px_status s = check_batch(in, "px_gather in");
    if (s != PX_OK) return s;
    s = check_batch(out, "px_gather out");
    if (s != PX_OK) return s;
    if (in->ncols != out->ncols || in->ncols < 1)
        return fail(PX_ERR_INVALID, "px_gather: %d input columns, %d output columns", in->ncols, out->ncols);
    for (int k = 0; k < in->ncols; ++k)
        if (in->cols[k].type != out->cols[k].type)
            return fail(PX_ERR_INVALID, "px_gather: column %d type differs between in and out", k);
    if (out->nrows > 0 && !d_idx) return fail(PX_ERR_INVALID, "px_gather: null d_idx");
    s = check_ws(d_ws, ws_bytes, kWsScratch, "px_gather");
    if (s != PX_OK) return s;
    if (out->nrows == 0) return PX_OK;
    GatherCols c;
    c.ncols = in->ncols;
    for (int k = 0; k < in->ncols; ++k) {
        c.width[k] = in->cols[k].type;
        c.in[k] = in->cols[k].data;
        c.out[k] = out->cols[k].data;
    }
    const int64_t ntiles = cdiv(out->nrows, static_cast<int64_t>(kThreads) * kItems);
    const unsigned grid = static_cast<unsigned>(std::min<int64_t>(ntiles, static_cast<int64_t>(sm_count()) * 8));
    gather_kernel<<<grid, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        c, d_idx, d_n, out->nrows, in->nrows, &static_cast<WsHeader*>(d_ws)->status);
    note_launch();
    return check_launch("px_gather");
}
