// px_groupby_agg: HashAggregation (Sec. 3.2) in Single mode, or Partial mode per
// segment (partition) when segments are given; a Final merge is another call.
//
// Group key: the key columns (and the segment id) packed into one 64-bit code,
// each key biased by its sign bit so the code orders like the signed tuple.
// Each block is persistent over a contiguous range of positions and keeps a
// shared-memory open-addressing table of (code -> 64-bit accumulators).
// Rows of one warp that share a code are first combined with shuffles (peers from
// match_any), so a hot key costs one shared-memory update per warp, not 32.
// Codes that find no room in the block's table go to a global table in the
// workspace; at the end every block merges its table into the global one. Global
// slots are claimed with a CAS on a state word (empty -> claimed -> published),
// take the next output row index from a counter, and accumulate with 64-bit
// atomics straight into the output columns. All arithmetic is mod 2^64.
#include <algorithm>

#include "px_common.cuh"

namespace px {
namespace {

constexpr int kThreads = 512;
constexpr int kItems = 4;
constexpr int kTile = kThreads * kItems;
constexpr int kSmemProbes = 32;
constexpr size_t kSmemBudget = 96 * 1024;

struct Spec {
    int32_t nkeys, keybits, segbits, nsegs;
    int32_t key_w[PX_MAX_KEYS];
    const void* key_in[PX_MAX_KEYS];
    void* key_out[PX_MAX_KEYS];
    int32_t naggs;
    int32_t op[PX_MAX_AGGS];
    int32_t a_w[PX_MAX_AGGS], b_w[PX_MAX_AGGS];
    const void* a_in[PX_MAX_AGGS];
    const void* b_in[PX_MAX_AGGS];
    int64_t* agg_out[PX_MAX_AGGS];
};

struct GTable {
    uint32_t* state;              // 0 empty, 1 claimed, 2 published
    unsigned long long* key;
    int32_t* gidx;                // output row of the group, -1 past capacity
    unsigned long long* ngroups;  // groups claimed so far
    uint32_t mask;
};

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t bits_mask(int bits) { return bits >= 64 ? ~0ull : ((1ull << bits) - 1); }

__device__ __forceinline__ uint64_t encode(const Spec& sp, int64_t row, int q) {
    uint64_t code = 0;
    for (int k = 0; k < sp.nkeys; ++k) {
        const int bits = 8 * sp.key_w[k];
        const uint64_t u = (static_cast<uint64_t>(load_int(sp.key_in[k], sp.key_w[k], row)) ^ (1ull << (bits - 1))) &
                           bits_mask(bits);
        code = bits >= 64 ? u : ((code << bits) | u);
    }
    if (sp.segbits) code |= static_cast<uint64_t>(q) << sp.keybits;
    return code;
}

__device__ __forceinline__ void write_group(const Spec& sp, uint64_t code, int32_t gi, int32_t* out_seg) {
    int shift = sp.keybits;
    for (int k = 0; k < sp.nkeys; ++k) {
        const int bits = 8 * sp.key_w[k];
        shift -= bits;
        const uint64_t u = (code >> shift) & bits_mask(bits);
        // u = raw ^ sb; sign-extending raw is (raw ^ sb) - sb = u - sb.
        const uint64_t sb = 1ull << (bits - 1);
        const int64_t v = static_cast<int64_t>(u - sb);
        store_int(sp.key_out[k], sp.key_w[k], gi, v);
    }
    if (out_seg) out_seg[gi] = sp.segbits ? static_cast<int32_t>(code >> sp.keybits) : 0;
}

// Output row of a group code, claiming a slot (and a row) on first sight.
__device__ int32_t global_group(const GTable& g, const Spec& sp, uint64_t code, int64_t max_groups, int32_t* out_seg,
                                int32_t* status) {
    uint32_t s = static_cast<uint32_t>(fmix64(code)) & g.mask;
    for (uint32_t probe = 0; probe <= g.mask; ++probe) {
        uint32_t st = ld_acquire_u32(&g.state[s]);
        if (st == 0) {
            st = atomicCAS(&g.state[s], 0u, 1u);
            if (st == 0) {
                const unsigned long long idx = atomicAdd(g.ngroups, 1ull);
                const int32_t gi = idx < static_cast<unsigned long long>(max_groups) ? static_cast<int32_t>(idx) : -1;
                g.key[s] = code;
                g.gidx[s] = gi;
                if (gi >= 0) write_group(sp, code, gi, out_seg);
                else set_status(status, PX_ERR_CAPACITY);
                __threadfence();
                atomicExch(&g.state[s], 2u);
                return gi;
            }
        }
        uint32_t spins = 0;
        while (st == 1) {
            if (++spins > kSpinLimit) {
                set_status(status, PX_ERR_TIMEOUT);
                return -1;
            }
            __nanosleep(32);
            st = ld_acquire_u32(&g.state[s]);
        }
        if (g.key[s] == code) return g.gidx[s];
        s = (s + 1) & g.mask;
    }
    set_status(status, PX_ERR_TABLE_FULL);
    return -1;
}

__device__ __forceinline__ void global_add(const GTable& g, const Spec& sp, uint64_t code, const uint64_t* v,
                                           int64_t max_groups, int32_t* out_seg, int32_t* status) {
    const int32_t gi = global_group(g, sp, code, max_groups, out_seg, status);
    if (gi < 0) return;
    for (int a = 0; a < sp.naggs; ++a)
        atomicAdd(reinterpret_cast<unsigned long long*>(&sp.agg_out[a][gi]), static_cast<unsigned long long>(v[a]));
}

// Slot of `code` in the block's table, inserting it if absent; -1 if no room
// within kSmemProbes probes.
__device__ __forceinline__ int smem_slot(uint32_t* s_state, unsigned long long* s_key, uint32_t smask, uint64_t code,
                                         int32_t* status) {
    uint32_t s = static_cast<uint32_t>(fmix64(code)) & smask;
    for (int probe = 0; probe < kSmemProbes; ++probe) {
        volatile uint32_t* vs = &s_state[s];
        uint32_t st = *vs;
        if (st == 0) {
            st = atomicCAS(&s_state[s], 0u, 1u);
            if (st == 0) {
                s_key[s] = code;
                __threadfence_block();
                *vs = 2u;
                return static_cast<int>(s);
            }
        }
        uint32_t spins = 0;
        while (st == 1) {
            if (++spins > kSpinLimit) {
                set_status(status, PX_ERR_TIMEOUT);
                return -1;
            }
            st = *vs;
        }
        __threadfence_block();
        if (static_cast<volatile unsigned long long*>(s_key)[s] == code) return static_cast<int>(s);
        s = (s + 1) & smask;
    }
    return -1;
}

__global__ void __launch_bounds__(kThreads)
groupby_kernel(Spec sp, const int32_t* __restrict__ sel, const int64_t* __restrict__ d_n, int64_t ncap,
               const int64_t* __restrict__ d_seg, GTable g, int64_t max_groups, int32_t* __restrict__ out_seg,
               int32_t* status, uint32_t sslots) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* s_acc = reinterpret_cast<unsigned long long*>(smem);      // naggs x sslots
    unsigned long long* s_key = s_acc + static_cast<size_t>(sp.naggs) * sslots;  // sslots
    uint32_t* s_state = reinterpret_cast<uint32_t*>(s_key + sslots);             // sslots
    const uint32_t smask = sslots - 1;
    const int tid = threadIdx.x, lane = tid & 31;
    for (uint32_t s = tid; s < sslots; s += kThreads) s_state[s] = 0;
    for (uint32_t s = tid; s < sslots * sp.naggs; s += kThreads) s_acc[s] = 0;
    __syncthreads();

    const int64_t n = actual_rows(d_n, ncap);
    const int64_t chunk = cdiv(cdiv(n, gridDim.x), kTile) * kTile;
    const int64_t cb = static_cast<int64_t>(blockIdx.x) * chunk;
    const int64_t ce = n < cb + chunk ? n : cb + chunk;
    for (int64_t tb = cb; tb < ce; tb += kTile) {
#pragma unroll 1
        for (int i = 0; i < kItems; ++i) {
            const int64_t j = tb + i * kThreads + tid;
            const bool valid = j < ce;
            uint64_t code = 0;
            uint64_t v[PX_MAX_AGGS];
            for (int a = 0; a < PX_MAX_AGGS; ++a) v[a] = 0;
            if (valid) {
                const int64_t r = sel ? static_cast<int64_t>(sel[j]) : j;
                const int q = sp.nsegs > 1 ? seg_of(d_seg, sp.nsegs, j) : 0;
                code = encode(sp, r, q);
                for (int a = 0; a < sp.naggs; ++a) {
                    if (sp.op[a] == PX_COUNT) {
                        v[a] = 1;
                    } else {
                        const uint64_t x = static_cast<uint64_t>(load_int(sp.a_in[a], sp.a_w[a], r));
                        v[a] = sp.op[a] == PX_SUM ? x
                                                  : x * static_cast<uint64_t>(load_int(sp.b_in[a], sp.b_w[a], r));
                    }
                }
            }
            const uint32_t vmask = __ballot_sync(FULL, valid);
            if (vmask == 0) continue;
            const uint32_t peers = __match_any_sync(FULL, code) & vmask;
            bool lead;
            if (vmask == FULL && peers == FULL) {
                // Whole warp on one group: butterfly reduction, lane 0 updates.
                for (int a = 0; a < sp.naggs; ++a) v[a] = warp_sum(v[a]);
                lead = (lane == 0);
            } else {
                // Each group's lowest lane gathers its peers' values.
                const int leader = valid ? __ffs(peers) - 1 : -1;
                lead = valid && lane == leader;
                uint32_t rest = lead ? (peers & ~(1u << lane)) : 0u;
                const int maxc = __reduce_max_sync(FULL, valid ? __popc(peers) : 0);
                for (int it = 1; it < maxc; ++it) {
                    const int src = rest ? __ffs(rest) - 1 : lane;
                    for (int a = 0; a < sp.naggs; ++a) {
                        const uint64_t x = __shfl_sync(FULL, v[a], src);
                        if (rest) v[a] += x;
                    }
                    if (rest) rest &= rest - 1;
                }
            }
            if (lead) {
                const int s = smem_slot(s_state, s_key, smask, code, status);
                if (s >= 0) {
                    for (int a = 0; a < sp.naggs; ++a) atomicAdd(&s_acc[static_cast<size_t>(a) * sslots + s], v[a]);
                } else {
                    global_add(g, sp, code, v, max_groups, out_seg, status);
                }
            }
        }
    }
    __syncthreads();
    // Merge this block's table into the global one.
    for (uint32_t s = tid; s < sslots; s += kThreads) {
        if (s_state[s] != 2) continue;
        uint64_t v[PX_MAX_AGGS];
        for (int a = 0; a < sp.naggs; ++a) v[a] = s_acc[static_cast<size_t>(a) * sslots + s];
        global_add(g, sp, s_key[s], v, max_groups, out_seg, status);
    }
}

uint32_t gtable_slots(int64_t max_groups) {
    uint64_t G = 1024;
    while (G < 2 * static_cast<uint64_t>(max_groups)) G <<= 1;
    return static_cast<uint32_t>(G);
}

uint32_t smem_slots(int naggs) {
    uint32_t s = 8192;
    while (s > 64 && static_cast<size_t>(s) * (12 + 8 * static_cast<size_t>(naggs)) > kSmemBudget) s >>= 1;
    return s;
}

int num_sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace
}  // namespace px

using namespace px;

extern "C" {

size_t px_groupby_ws_bytes(int64_t nrows, int64_t max_groups) {
    (void)nrows;
    if (max_groups < 1) max_groups = 1;
    const size_t G = gtable_slots(max_groups);
    return kWsScratch + 256 + align_up(4 * G, 256) + align_up(8 * G, 256) + align_up(4 * G, 256);
}

px_status px_groupby_agg(const px_batch* in, const int32_t* key_cols, int32_t nkeys, const px_agg* aggs,
                         int32_t naggs, const int32_t* d_sel, const int64_t* d_nsel, const int64_t* d_seg,
                         int32_t nsegs, int64_t max_groups, const px_batch* out, int32_t* d_out_seg,
                         int64_t* d_ngroups, void* d_ws, size_t ws_bytes, void* stream) {
    set_error("");
    px_status s = check_batch(in, "px_groupby_agg in");
    if (s != PX_OK) return s;
    if (nkeys < 1 || nkeys > PX_MAX_KEYS || !key_cols)
        return fail(PX_ERR_UNSUPPORTED, "px_groupby_agg: nkeys %d outside [1, %d]", nkeys, PX_MAX_KEYS);
    if (naggs < 0 || naggs > PX_MAX_AGGS || (naggs > 0 && !aggs))
        return fail(PX_ERR_UNSUPPORTED, "px_groupby_agg: naggs %d outside [0, %d]", naggs, PX_MAX_AGGS);
    if ((d_sel == nullptr) != (d_nsel == nullptr))
        return fail(PX_ERR_INVALID, "px_groupby_agg: d_sel and d_nsel must be given together");
    if (nsegs < 0 || nsegs > PX_MAX_SEGS)
        return fail(PX_ERR_UNSUPPORTED, "px_groupby_agg: nsegs %d outside [0, %d]", nsegs, PX_MAX_SEGS);
    if ((nsegs > 0) != (d_seg != nullptr))
        return fail(PX_ERR_INVALID, "px_groupby_agg: d_seg must be given exactly when nsegs > 0");
    if (max_groups < 1 || max_groups > INT32_MAX)
        return fail(PX_ERR_INVALID, "px_groupby_agg: max_groups %lld", (long long)max_groups);
    if (!d_ngroups) return fail(PX_ERR_INVALID, "px_groupby_agg: null d_ngroups");
    s = check_batch(out, "px_groupby_agg out");
    if (s != PX_OK) return s;
    if (out->ncols != nkeys + naggs)
        return fail(PX_ERR_INVALID, "px_groupby_agg: out has %d columns, %d expected", out->ncols, nkeys + naggs);
    if (out->nrows < max_groups)
        return fail(PX_ERR_INVALID, "px_groupby_agg: out capacity %lld below max_groups", (long long)out->nrows);
    Spec sp;
    sp.nkeys = nkeys;
    sp.keybits = 0;
    for (int k = 0; k < nkeys; ++k) {
        if (key_cols[k] < 0 || key_cols[k] >= in->ncols)
            return fail(PX_ERR_INVALID, "px_groupby_agg: key column %d out of range", key_cols[k]);
        const px_col& c = in->cols[key_cols[k]];
        if (out->cols[k].type != c.type)
            return fail(PX_ERR_INVALID, "px_groupby_agg: out key column %d type differs from input key", k);
        sp.key_w[k] = c.type;
        sp.key_in[k] = c.data;
        sp.key_out[k] = out->cols[k].data;
        sp.keybits += 8 * c.type;
    }
    sp.nsegs = nsegs;
    sp.segbits = 0;
    while (nsegs > 1 && (1ll << sp.segbits) < nsegs) ++sp.segbits;
    if (sp.keybits + sp.segbits > 64)
        return fail(PX_ERR_UNSUPPORTED, "px_groupby_agg: %d key bits + %d segment bits exceed 64", sp.keybits,
                    sp.segbits);
    sp.naggs = naggs;
    for (int a = 0; a < naggs; ++a) {
        const px_agg& ag = aggs[a];
        if (ag.op != PX_COUNT && ag.op != PX_SUM && ag.op != PX_SUM_MUL)
            return fail(PX_ERR_INVALID, "px_groupby_agg: aggregate %d has unknown op %d", a, ag.op);
        sp.op[a] = ag.op;
        sp.a_w[a] = sp.b_w[a] = 8;
        sp.a_in[a] = sp.b_in[a] = nullptr;
        if (ag.op != PX_COUNT) {
            if (ag.a < 0 || ag.a >= in->ncols) return fail(PX_ERR_INVALID, "px_groupby_agg: aggregate %d column a", a);
            sp.a_w[a] = in->cols[ag.a].type;
            sp.a_in[a] = in->cols[ag.a].data;
        }
        if (ag.op == PX_SUM_MUL) {
            if (ag.b < 0 || ag.b >= in->ncols) return fail(PX_ERR_INVALID, "px_groupby_agg: aggregate %d column b", a);
            sp.b_w[a] = in->cols[ag.b].type;
            sp.b_in[a] = in->cols[ag.b].data;
        }
        if (out->cols[nkeys + a].type != PX_I64)
            return fail(PX_ERR_INVALID, "px_groupby_agg: aggregate output column %d must be PX_I64", nkeys + a);
        sp.agg_out[a] = static_cast<int64_t*>(out->cols[nkeys + a].data);
    }
    s = check_ws(d_ws, ws_bytes, px_groupby_ws_bytes(in->nrows, max_groups), "px_groupby_agg");
    if (s != PX_OK) return s;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t G = gtable_slots(max_groups);
    char* base = static_cast<char*>(d_ws) + kWsScratch;
    GTable g;
    g.ngroups = reinterpret_cast<unsigned long long*>(base);
    g.state = reinterpret_cast<uint32_t*>(base + 256);
    g.key = reinterpret_cast<unsigned long long*>(base + 256 + align_up(4ull * G, 256));
    g.gidx = reinterpret_cast<int32_t*>(base + 256 + align_up(4ull * G, 256) + align_up(8ull * G, 256));
    g.mask = G - 1;
    cudaMemsetAsync(base, 0, 256 + 4ull * G, st);
    for (int a = 0; a < naggs; ++a) cudaMemsetAsync(sp.agg_out[a], 0, 8ull * max_groups, st);
    const int64_t ncap = in->nrows;
    if (ncap > 0) {
        const uint32_t sslots = smem_slots(naggs);
        const size_t smem = static_cast<size_t>(sslots) * (12 + 8 * static_cast<size_t>(naggs));
        cudaFuncSetAttribute(groupby_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, groupby_kernel, kThreads, smem);
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(cdiv(ncap, kTile),
                                                                    static_cast<int64_t>(num_sms()) * std::max(1, per_sm)));
        const int64_t* d_n = d_sel ? d_nsel : in->d_nrows;
        groupby_kernel<<<static_cast<unsigned>(grid), kThreads, smem, st>>>(
            sp, d_sel, d_n, ncap, d_seg, g, max_groups, d_out_seg, &static_cast<WsHeader*>(d_ws)->status, sslots);
        note_launch();
        if ((s = check_launch("px_groupby_agg")) != PX_OK) return s;
    }
    cudaMemcpyAsync(d_ngroups, g.ngroups, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    return check_launch("px_groupby_agg count");
}

}  // extern "C"
