// px_groupby_agg: HashAggregation (Sec. 3.2) in Single mode, or Partial mode per
// segment (partition) when segments are given; a Final merge is another call.
//
// Group key: the key columns (and the segment id) packed into one 64-bit code,
// each key biased by its sign bit so the code orders like the signed tuple.
// Each block is persistent over a contiguous range of positions, which it walks
// segment by segment. Per segment it aggregates into a block-local table and
// merges that table into the global result when the segment ends (codes of a
// finished segment never recur in the block's range, so the table starts empty
// for the next one). The block-local table is either
//   * dense: when the caller's key-range statistic makes the key space small,
//     shared-memory arrays indexed by the key offset, replicated per warp when
//     they fit (fewer same-address atomics); rows outside the range take the
//     global path; or
//   * hashed: an open-addressing shared-memory table (code -> accumulators);
//     codes that find no room within a few probes take the global path.
// Rows of one warp with equal codes are first combined with shuffles (peers from
// match_any), so a hot key costs one shared-memory update per warp, not 32.
// The global table lives in the workspace: slots are claimed with a CAS on a
// state word (empty -> claimed -> published), take the next output row from a
// counter, and accumulate with 64-bit reductions straight into the output columns.
// All arithmetic is mod 2^64. Every thread loads all of its rows' inputs for a
// tile before aggregating any of them, so each thread keeps many loads in flight.
#include <algorithm>

#include "px_common.cuh"
#include "px_table.cuh"

namespace px {
namespace {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 4;
constexpr int kTile = kThreads * kItems;
constexpr int kSmemProbes = 8;
constexpr int kMajority = 6;  // smallest group worth a warp reduction
constexpr size_t kSmemBudget = 192 * 1024;

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
    // dense mode: per replica, SUM-like aggregates in u64 arrays [n64][D], COUNT
    // aggregates in u32 arrays [n32][D] (a block counts < 2^32 rows per segment),
    // then an occupancy bitmap when there is no COUNT.
    int32_t dense;      // 1: dense block arrays
    int32_t reps;       // replicas: kThreads (one per thread, plain adds) or 1..kWarps (warp w: w % reps)
    int32_t count_agg;  // a COUNT aggregate marks occupancy; -1: use the bitmap
    uint32_t D;         // dense slots per replica
    int32_t n64, n32;
    int32_t kind[PX_MAX_AGGS];  // 0: u64 array, 1: u32 array
    int32_t slot[PX_MAX_AGGS];  // index of the aggregate's array within its kind
    uint32_t rep_bytes;         // bytes per replica
    int64_t lo[PX_MAX_KEYS];
    uint64_t span[PX_MAX_KEYS];
    // dense global result (when the whole (segment, key) space fits max_groups)
    int32_t dglobal;
    int32_t direct;               // rows update the dense global array directly (no block arrays)
    uint64_t E;                   // entries: max(nsegs, 1) * D
    unsigned long long* dg_acc;   // [naggs][E]
    uint8_t* dg_occ;              // [E] occupancy flags, 1 where the entry has rows (only without COUNT)
    // fused probe (px_join_probe_agg): the key of position j is group[build row of
    // fk[j] in segment q of the table], or no group when fk[j] has no match
    const int64_t* probe_fk;
    TableView probe_t;
    const void* group_col;
    int32_t group_w;
    int64_t nbuild;
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

// Group code of key values k0 (, k1) (sign-extended) in segment q.
__device__ __forceinline__ uint64_t compose(const Spec& sp, int64_t k0, int64_t k1, int q) {
    const int b0 = 8 * sp.key_w[0];
    uint64_t code = (static_cast<uint64_t>(k0) ^ (1ull << (b0 - 1))) & bits_mask(b0);
    if (sp.nkeys > 1) {
        const int b1 = 8 * sp.key_w[1];
        code = (code << b1) | ((static_cast<uint64_t>(k1) ^ (1ull << (b1 - 1))) & bits_mask(b1));
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
        store_int(sp.key_out[k], sp.key_w[k], gi, static_cast<int64_t>(u - sb));
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
                if (gi >= 0) {
                    write_group(sp, code, gi, out_seg);
                    // The row's accumulators start at zero (an output row may hold an
                    // earlier call's value when calls accumulate into one table).
                    for (int a = 0; a < sp.naggs; ++a) sp.agg_out[a][gi] = 0;
                } else {
                    set_status(status, PX_ERR_CAPACITY);
                }
                __threadfence();
                atomicExch(&g.state[s], 2u);
                return gi;
            }
            // The CAS lost to another claimer; it carries no acquire ordering, so
            // read the state again with one before trusting key and gidx.
            st = ld_acquire_u32(&g.state[s]);
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
        red_add_global(reinterpret_cast<unsigned long long*>(&sp.agg_out[a][gi]), static_cast<unsigned long long>(v[a]));
}

// Slot of `code` in the block's hash table, inserting it if absent; -1 if no
// room within kSmemProbes probes.
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

struct Smem {
    // dense: replicas of rep_bytes each (see Spec)
    unsigned char* rep0;
    uint32_t occ_words;
    // hashed: low words [naggs][S], high words [naggs][S], key[S], state[S]
    uint32_t* h_lo;
    uint32_t* h_hi;
    unsigned long long* h_key;
    uint32_t* h_state;
    uint32_t S;
};

// A replica holds each 64-bit sum as two 32-bit words, low words [n64][D] then
// high words [n64][D], so every update is a native 32-bit shared atomic: a 64-bit
// shared atomicAdd retries under contention and collapses on hot keys.
__device__ __forceinline__ uint32_t* rep_lo(const Spec& sp, const Smem& m, int r) {
    return reinterpret_cast<uint32_t*>(m.rep0 + static_cast<size_t>(r) * sp.rep_bytes);
}
__device__ __forceinline__ uint32_t* rep_hi(const Spec& sp, const Smem& m, int r) {
    return rep_lo(sp, m, r) + static_cast<size_t>(sp.n64) * sp.D;
}
__device__ __forceinline__ uint32_t* rep_u32(const Spec& sp, const Smem& m, int r) {
    return rep_lo(sp, m, r) + 2 * static_cast<size_t>(sp.n64) * sp.D;
}

// Adds x (mod 2^64) to the 64-bit value held as words lo/hi: the returned old low
// word tells whether the low addition wrapped; the high word changes only when x
// has high bits or the low word carried. Exact once all updates have landed.
__device__ __forceinline__ void add_split_atomic(uint32_t* lo, uint32_t* hi, uint64_t x) {
    const uint32_t xl = static_cast<uint32_t>(x), xh = static_cast<uint32_t>(x >> 32);
    const uint32_t old = atomicAdd(lo, xl);
    const uint32_t add_hi = xh + (old + xl < old ? 1u : 0u);
    if (add_hi) red_add_shared(hi, add_hi);
}
__device__ __forceinline__ void add_split(uint32_t* lo, uint32_t* hi, uint64_t x) {
    const uint32_t xl = static_cast<uint32_t>(x), old = *lo;
    *lo = old + xl;
    *hi += static_cast<uint32_t>(x >> 32) + (old + xl < old ? 1u : 0u);
}
__device__ __forceinline__ uint32_t* rep_occ(const Spec& sp, const Smem& m, int r) {
    return rep_u32(sp, m, r) + static_cast<size_t>(sp.n32) * sp.D;
}

__device__ __forceinline__ void clear_block_table(const Spec& sp, const Smem& m) {
    if (sp.dense) {
        uint32_t* w = reinterpret_cast<uint32_t*>(m.rep0);
        const uint32_t nw = static_cast<uint32_t>(sp.reps) * sp.rep_bytes / 4;
        for (uint32_t i = threadIdx.x; i < nw; i += kThreads) w[i] = 0;
    } else {
        for (uint32_t s = threadIdx.x; s < m.S; s += kThreads) m.h_state[s] = 0;
        for (uint32_t s = threadIdx.x; s < m.S * sp.naggs; s += kThreads) m.h_lo[s] = m.h_hi[s] = 0;
    }
}

// Merge the block table (segment q) into the global table and clear it.
__device__ void flush_block_table(const Spec& sp, const Smem& m, int q, const GTable& g, int64_t max_groups,
                                  int32_t* out_seg, int32_t* status) {
    __syncthreads();
    // A warp per slot (lanes over the replicas, then a warp sum) when there are few
    // slots for many replicas: a thread per slot would walk every replica alone
    // while the rest of the block waits at the barrier. With many slots the thread
    // per slot keeps every thread busy and wins (a warp sum costs ~12 thread-slot
    // steps).
    const bool warp_flush = sp.dense && (sp.D + kWarps - 1) / kWarps * 12 <
                                            (sp.D + kThreads - 1) / kThreads * static_cast<uint32_t>(sp.reps);
    if (warp_flush) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (uint32_t d = warp; d < sp.D; d += kWarps) {
            uint64_t v[PX_MAX_AGGS];
            bool occ = false;
            for (int a = 0; a < sp.naggs; ++a) v[a] = 0;
            for (int r = lane; r < sp.reps; r += 32) {
                uint32_t* LO = rep_lo(sp, m, r);
                uint32_t* HI = rep_hi(sp, m, r);
                uint32_t* A32 = rep_u32(sp, m, r);
                for (int a = 0; a < sp.naggs; ++a) {
                    if (sp.kind[a] == 0) {
                        const size_t o = static_cast<size_t>(sp.slot[a]) * sp.D + d;
                        v[a] += (static_cast<uint64_t>(HI[o]) << 32) | LO[o];
                        LO[o] = 0;
                        HI[o] = 0;
                    } else {
                        uint32_t* p = &A32[static_cast<size_t>(sp.slot[a]) * sp.D + d];
                        v[a] += *p;
                        *p = 0;
                    }
                }
                if (sp.count_agg < 0) occ |= ((rep_occ(sp, m, r)[d / 32] >> (d % 32)) & 1u) != 0;
            }
            for (int a = 0; a < sp.naggs; ++a) v[a] = warp_sum(v[a]);
            occ = __any_sync(FULL, occ);
            if (sp.count_agg >= 0) occ = v[sp.count_agg] != 0;
            if (!occ || lane != 0) continue;
            if (sp.dglobal) {
                const uint64_t e = static_cast<uint64_t>(q) * sp.D + d;
                for (int a = 0; a < sp.naggs; ++a)
                    red_add_global(&sp.dg_acc[a * sp.E + e], static_cast<unsigned long long>(v[a]));
                if (sp.count_agg < 0) sp.dg_occ[e] = 1;
                continue;
            }
            const int64_t k0 = sp.lo[0] + static_cast<int64_t>(d / sp.span[1]);
            const int64_t k1 = sp.nkeys > 1 ? sp.lo[1] + static_cast<int64_t>(d % sp.span[1]) : 0;
            global_add(g, sp, compose(sp, k0, k1, q), v, max_groups, out_seg, status);
        }
        __syncthreads();
        if (sp.count_agg < 0)
            for (uint32_t i = threadIdx.x; i < sp.reps * m.occ_words; i += kThreads)
                rep_occ(sp, m, i / m.occ_words)[i % m.occ_words] = 0;
    } else if (sp.dense) {
        for (uint32_t d = threadIdx.x; d < sp.D; d += kThreads) {
            uint64_t v[PX_MAX_AGGS];
            bool occ = false;
            for (int a = 0; a < sp.naggs; ++a) v[a] = 0;
            for (int r = 0; r < sp.reps; ++r) {
                uint32_t* LO = rep_lo(sp, m, r);
                uint32_t* HI = rep_hi(sp, m, r);
                uint32_t* A32 = rep_u32(sp, m, r);
                for (int a = 0; a < sp.naggs; ++a) {
                    if (sp.kind[a] == 0) {
                        const size_t o = static_cast<size_t>(sp.slot[a]) * sp.D + d;
                        v[a] += (static_cast<uint64_t>(HI[o]) << 32) | LO[o];
                        LO[o] = 0;
                        HI[o] = 0;
                    } else {
                        uint32_t* p = &A32[static_cast<size_t>(sp.slot[a]) * sp.D + d];
                        v[a] += *p;
                        *p = 0;
                    }
                }
                if (sp.count_agg < 0) occ |= ((rep_occ(sp, m, r)[d / 32] >> (d % 32)) & 1u) != 0;
            }
            if (sp.count_agg >= 0) occ = v[sp.count_agg] != 0;
            if (!occ) continue;
            if (sp.dglobal) {
                // Dense global array: entry (segment q, slot d); no hashing, no claim.
                const uint64_t e = static_cast<uint64_t>(q) * sp.D + d;
                for (int a = 0; a < sp.naggs; ++a)
                    red_add_global(&sp.dg_acc[a * sp.E + e], static_cast<unsigned long long>(v[a]));
                if (sp.count_agg < 0) sp.dg_occ[e] = 1;  // every writer stores the same value
                continue;
            }
            const int64_t k0 = sp.lo[0] + static_cast<int64_t>(d / sp.span[1]);
            const int64_t k1 = sp.nkeys > 1 ? sp.lo[1] + static_cast<int64_t>(d % sp.span[1]) : 0;
            global_add(g, sp, compose(sp, k0, k1, q), v, max_groups, out_seg, status);
        }
        __syncthreads();
        if (sp.count_agg < 0)
            for (uint32_t i = threadIdx.x; i < sp.reps * m.occ_words; i += kThreads)
                rep_occ(sp, m, i / m.occ_words)[i % m.occ_words] = 0;
    } else {
        for (uint32_t s = threadIdx.x; s < m.S; s += kThreads) {
            if (m.h_state[s] == 2) {
                uint64_t v[PX_MAX_AGGS];
                for (int a = 0; a < sp.naggs; ++a) {
                    const size_t o = static_cast<size_t>(a) * m.S + s;
                    v[a] = (static_cast<uint64_t>(m.h_hi[o]) << 32) | m.h_lo[o];
                    m.h_lo[o] = m.h_hi[o] = 0;
                }
                global_add(g, sp, m.h_key[s], v, max_groups, out_seg, status);
            }
            m.h_state[s] = 0;
        }
    }
    __syncthreads();
}

constexpr uint32_t kIdxNone = 0xffffffffu;   // no row at this item
constexpr uint32_t kIdxOutside = 0xfffffffeu;  // key outside the dense range

// v[i] = column value at row[i] (sign-extended), 0 where row[i] < 0. One type
// switch per column, then kItems independent loads.
template <typename T>
__device__ __forceinline__ void load_col_t(const void* p, const int32_t* row, int64_t* v) {
#pragma unroll
    for (int i = 0; i < kItems; ++i) v[i] = row[i] >= 0 ? static_cast<int64_t>(static_cast<const T*>(p)[row[i]]) : 0;
}
__device__ __forceinline__ void load_col(const void* p, int w, const int32_t* row, int64_t* v) {
    if (w == 8) load_col_t<int64_t>(p, row, v);
    else if (w == 4) load_col_t<int32_t>(p, row, v);
    else load_col_t<int8_t>(p, row, v);
}

// Dense-mode aggregation of positions [a0, a1) of segment q: keys become slot
// indices at load time, each aggregate is applied with one atomic per row (or a
// plain add into the thread's private replica), rows outside the key range take
// the global path afterwards.
// DIRECT: no block arrays; every in-range row (or warp-combined hot key) adds
// straight into the dense global array with 64-bit global reductions. Chosen for
// inputs with few rows per entry, where block arrays would cost more to clear
// and flush than they save (a Final merge of Partial results, say).
// PROBE: the key of each position comes from the fused join probe (see Spec).
template <int NA, bool DIRECT, bool PROBE>
__device__ void aggregate_range_dense(const Spec& sp, const Smem& m, const int32_t* __restrict__ sel, int64_t a0,
                                      int64_t a1, int q, const GTable& g, int64_t max_groups, int32_t* out_seg,
                                      int32_t* status) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool private_rep = !DIRECT && sp.reps == kThreads;
    const int rep = private_rep ? tid : warp % sp.reps;
    uint32_t* const LO = DIRECT ? nullptr : rep_lo(sp, m, rep);
    uint32_t* const HI = DIRECT ? nullptr : rep_hi(sp, m, rep);
    uint32_t* const A32 = DIRECT ? nullptr : rep_u32(sp, m, rep);
    uint32_t* const OCC = DIRECT ? nullptr : rep_occ(sp, m, rep);
    const uint64_t ebase = static_cast<uint64_t>(q) * sp.D;
    SegGeom geo = {};
    bool group_in_table = false;  // PROBE: the table holds the group column beside the keys
    if (PROBE) {
        geo = seg_geom(sp.probe_t, q);
        group_in_table = sp.probe_t.hdr->pay_src == sp.group_col && sp.probe_t.hdr->pay_w == sp.group_w;
    }
    for (int64_t tb = a0; tb < a1; tb += kTile) {
        int32_t row[kItems];
        uint32_t idx[kItems];
        int64_t pkey[kItems];  // PROBE: the gathered group key
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int64_t j = tb + i * kThreads + tid;
            row[i] = j < a1 ? (sel ? sel[j] : static_cast<int32_t>(j)) : -1;
        }
        if (PROBE) {
            // Join probe of every position: its key's home bucket (one sector: keys,
            // rows and copied payload values), a walk on in the rare case that bucket
            // is full without it, then the group key: the copied payload value when the
            // table holds the group column, else gathered from the build column.
            int64_t fkv[kItems];
            BucketRegs bv[kItems];
#pragma unroll
            for (int i = 0; i < kItems; ++i) fkv[i] = row[i] >= 0 ? sp.probe_fk[row[i]] : kEmpty;
            const Bucket* const segb = sp.probe_t.bk + geo.b0;
            uint32_t hb[kItems];
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                hb[i] = home_bucket(static_cast<uint64_t>(fkv[i]), geo.nb);
                bv[i] = load_bucket(segb + hb[i]);  // hb < nb: inside the segment
            }
            int32_t brow[kItems], bpay[kItems];
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                brow[i] = -1;
                bpay[i] = 0;
                if (fkv[i] == kEmpty) continue;
                bool end;
                int l = bucket_find(bv[i], fkv[i], &end);
                if (l < 0 && !end) l = walk_find(segb, geo.nb, hb[i], fkv[i], &bv[i]);
                if (l >= 0) {
                    brow[i] = bucket_row(bv[i], l);
                    bpay[i] = bucket_pay(bv[i], l);
                }
            }
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                pkey[i] = brow[i] < 0 ? 0
                                      : (group_in_table ? static_cast<int64_t>(bpay[i])
                                                           : load_int(sp.group_col, sp.group_w, brow[i]));
                const uint64_t o0 = static_cast<uint64_t>(pkey[i] - sp.lo[0]);
                idx[i] = brow[i] < 0 ? kIdxNone : (o0 < sp.span[0] ? static_cast<uint32_t>(o0) : kIdxOutside);
            }
        } else {
            int64_t k0[kItems], k1[kItems];
            load_col(sp.key_in[0], sp.key_w[0], row, k0);
            if (sp.nkeys > 1) load_col(sp.key_in[1], sp.key_w[1], row, k1);
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                pkey[i] = 0;
                const uint64_t o0 = static_cast<uint64_t>(k0[i] - sp.lo[0]);
                const uint64_t o1 = sp.nkeys > 1 ? static_cast<uint64_t>(k1[i] - sp.lo[1]) : 0;
                idx[i] = row[i] < 0 ? kIdxNone
                                    : ((o0 < sp.span[0] && o1 < sp.span[1]) ? static_cast<uint32_t>(o0 * sp.span[1] + o1)
                                                                            : kIdxOutside);
            }
        }
        int64_t v[NA > 0 ? NA : 1][kItems];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            if (a >= sp.naggs) break;
            if (sp.op[a] == PX_COUNT) {
#pragma unroll
                for (int i = 0; i < kItems; ++i) v[a][i] = 1;
            } else {
                load_col(sp.a_in[a], sp.a_w[a], row, v[a]);
                if (sp.op[a] == PX_SUM_MUL) {
                    int64_t y[kItems];
                    load_col(sp.b_in[a], sp.b_w[a], row, y);
#pragma unroll
                    for (int i = 0; i < kItems; ++i)
                        v[a][i] = static_cast<int64_t>(static_cast<uint64_t>(v[a][i]) * static_cast<uint64_t>(y[i]));
                }
            }
        }
        // Hot keys: when lane 0's slot is shared by at least kMajority lanes, those
        // rows are summed across the warp (COUNT is the peer count; 64-bit sums are
        // three 32-bit warp reductions) and lane 0 applies them once (many lanes
        // on one address would serialise the shared-memory atomics).
        uint32_t apply[kItems];
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            apply[i] = idx[i];
            if (private_rep) continue;
            const uint32_t c0 = __shfl_sync(FULL, idx[i], 0);
            const uint32_t mm = __ballot_sync(FULL, idx[i] == c0);
            if (c0 < kIdxOutside && __popc(mm) >= kMajority) {
                const bool in = (mm >> lane) & 1u;
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    if (a >= sp.naggs) break;
                    // The probe-fed kernel keeps the shuffle butterfly: redux.sync's
                    // longer latency measured slower there.
                    const int64_t x = PROBE ? warp_sum(in ? v[a][i] : int64_t(0))
                                    : sp.op[a] == PX_COUNT
                                          ? static_cast<int64_t>(__popc(mm))
                                          : static_cast<int64_t>(warp_sum_u64(in ? static_cast<uint64_t>(v[a][i]) : 0));
                    if (lane == 0) v[a][i] = x;
                }
                if (in && lane != 0) apply[i] = kIdxNone;
            }
        }
        // Apply in-range rows.
        if (DIRECT) {
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                if (apply[i] >= kIdxOutside) continue;
                const uint64_t e = ebase + apply[i];
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    if (a >= sp.naggs) break;
                    red_add_global(&sp.dg_acc[a * sp.E + e], static_cast<unsigned long long>(v[a][i]));
                }
                if (sp.count_agg < 0) sp.dg_occ[e] = 1;  // every writer stores the same value
            }
        }
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            if (DIRECT || a >= sp.naggs) break;
            const size_t off = static_cast<size_t>(sp.slot[a]) * sp.D;
            if (sp.kind[a] == 0) {
#pragma unroll
                for (int i = 0; i < kItems; ++i) {
                    if (apply[i] >= kIdxOutside) continue;
                    if (private_rep) add_split(&LO[off + apply[i]], &HI[off + apply[i]], static_cast<uint64_t>(v[a][i]));
                    else add_split_atomic(&LO[off + apply[i]], &HI[off + apply[i]], static_cast<uint64_t>(v[a][i]));
                }
            } else {
#pragma unroll
                for (int i = 0; i < kItems; ++i) {
                    if (apply[i] >= kIdxOutside) continue;
                    if (private_rep) A32[off + apply[i]] += static_cast<uint32_t>(v[a][i]);
                    else red_add_shared(&A32[off + apply[i]], static_cast<uint32_t>(v[a][i]));
                }
            }
        }
        if (!DIRECT && sp.count_agg < 0) {
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                if (apply[i] >= kIdxOutside) continue;
                if (private_rep) OCC[apply[i] / 32] |= 1u << (apply[i] % 32);
                else red_or_shared(&OCC[apply[i] / 32], 1u << (apply[i] % 32));
            }
        }
        // Rows outside the key range (rare when the statistic is right): global path.
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            if (idx[i] != kIdxOutside) continue;
            const int64_t r = row[i];
            const int64_t k0 = PROBE ? pkey[i] : load_int(sp.key_in[0], sp.key_w[0], r);
            const int64_t k1 = !PROBE && sp.nkeys > 1 ? load_int(sp.key_in[1], sp.key_w[1], r) : 0;
            uint64_t full[PX_MAX_AGGS];
#pragma unroll
            for (int a = 0; a < NA; ++a) full[a] = static_cast<uint64_t>(v[a][i]);
            global_add(g, sp, compose(sp, k0, k1, q), full, max_groups, out_seg, status);
        }
    }
}

// Hash-mode aggregation of positions [a0, a1) of segment q into the block's
// shared-memory hash table; codes that find no room go to the global table. NA:
// number of aggregates when known at compile time (0..4), or PX_MAX_AGGS.
template <int NA>
__device__ void aggregate_range(const Spec& sp, const Smem& m, const int32_t* __restrict__ sel, int64_t a0, int64_t a1,
                                int q, const GTable& g, int64_t max_groups, int32_t* out_seg, int32_t* status) {
    const int tid = threadIdx.x, lane = tid & 31;
    for (int64_t tb = a0; tb < a1; tb += kTile) {
        int32_t row[kItems];
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int64_t j = tb + i * kThreads + tid;
            row[i] = j < a1 ? (sel ? sel[j] : static_cast<int32_t>(j)) : -1;
        }
        uint64_t code[kItems];
        {
            int64_t k0[kItems], k1[kItems];
            load_col(sp.key_in[0], sp.key_w[0], row, k0);
            if (sp.nkeys > 1) load_col(sp.key_in[1], sp.key_w[1], row, k1);
#pragma unroll
            for (int i = 0; i < kItems; ++i) code[i] = compose(sp, k0[i], sp.nkeys > 1 ? k1[i] : 0, q);
        }
        int64_t v[NA > 0 ? NA : 1][kItems];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            if (a >= sp.naggs) break;
            if (sp.op[a] == PX_COUNT) {
#pragma unroll
                for (int i = 0; i < kItems; ++i) v[a][i] = 1;
            } else {
                load_col(sp.a_in[a], sp.a_w[a], row, v[a]);
                if (sp.op[a] == PX_SUM_MUL) {
                    int64_t y[kItems];
                    load_col(sp.b_in[a], sp.b_w[a], row, y);
#pragma unroll
                    for (int i = 0; i < kItems; ++i)
                        v[a][i] = static_cast<int64_t>(static_cast<uint64_t>(v[a][i]) * static_cast<uint64_t>(y[i]));
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const bool valid = row[i] >= 0;
            // Hot keys: lane 0's code shared by >= kMajority lanes is summed across
            // the warp and applied once by lane 0.
            bool lead = valid;
            const uint64_t c0 = __shfl_sync(FULL, code[i], 0);
            const uint32_t mm = __ballot_sync(FULL, valid && code[i] == c0);
            if ((mm & 1u) && __popc(mm) >= kMajority) {
                const bool in = (mm >> lane) & 1u;
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    if (a >= sp.naggs) break;
                    const int64_t x = sp.op[a] == PX_COUNT
                                          ? static_cast<int64_t>(__popc(mm))
                                          : static_cast<int64_t>(warp_sum_u64(in ? static_cast<uint64_t>(v[a][i]) : 0));
                    if (lane == 0) v[a][i] = x;
                }
                lead = valid && (!in || lane == 0);
            }
            if (!lead) continue;
            const int s = smem_slot(m.h_state, m.h_key, m.S - 1, code[i], status);
            if (s >= 0) {
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    if (a >= sp.naggs) break;
                    const size_t o = static_cast<size_t>(a) * m.S + s;
                    add_split_atomic(&m.h_lo[o], &m.h_hi[o], static_cast<uint64_t>(v[a][i]));
                }
            } else {
                uint64_t full[PX_MAX_AGGS];
#pragma unroll
                for (int a = 0; a < NA; ++a) full[a] = static_cast<uint64_t>(v[a][i]);
                global_add(g, sp, code[i], full, max_groups, out_seg, status);
            }
        }
    }
}

// Modes: kHashed, kDenseBlock (block arrays) and kDenseDirect (rows straight into
// the dense global array). MODE must agree with sp.dense / sp.direct: the modes are
// separate kernels so each gets its own register allocation.
constexpr int kHashed = 0, kDenseBlock = 1, kDenseDirect = 2;

template <int NA, int MODE, bool PROBE = false>
__global__ void __launch_bounds__(kThreads)
groupby_kernel(Spec sp, const int32_t* __restrict__ sel, const int64_t* __restrict__ d_n, int64_t ncap,
               const int64_t* __restrict__ d_seg, GTable g, int64_t max_groups, int32_t* __restrict__ out_seg,
               int32_t* status, uint32_t hash_slots) {
    extern __shared__ __align__(16) unsigned char smem[];
    Smem m = {};
    if (MODE == kDenseBlock) {
        m.rep0 = smem;
        m.occ_words = (sp.D + 31) / 32;
    } else if (MODE == kHashed) {
        m.S = hash_slots;
        m.h_lo = reinterpret_cast<uint32_t*>(smem);
        m.h_hi = m.h_lo + static_cast<size_t>(sp.naggs) * hash_slots;
        m.h_key = reinterpret_cast<unsigned long long*>(m.h_hi + static_cast<size_t>(sp.naggs) * hash_slots);
        m.h_state = reinterpret_cast<uint32_t*>(m.h_key + hash_slots);
    }
    if (MODE != kDenseDirect) {
        clear_block_table(sp, m);
        __syncthreads();
    }

    if (PROBE) {  // a table this call cannot use: no groups (uniform across the block)
        const TableHeader* h = sp.probe_t.hdr;
        const int S = sp.nsegs > 0 ? sp.nsegs : 1;
        if (h->magic != kMagic || h->nsegs != S || h->unique == 0 || h->nbuild > sp.nbuild) {
            if (blockIdx.x == 0 && threadIdx.x == 0)
                set_status(status, h->magic == kMagic && h->unique == 0 ? PX_ERR_UNSUPPORTED : PX_ERR_INVALID);
            return;
        }
    }
    const int64_t n = actual_rows(d_n, ncap);
    const int64_t chunk = cdiv(cdiv(n, gridDim.x), kTile) * kTile;
    const int64_t cb = static_cast<int64_t>(blockIdx.x) * chunk;
    const int64_t ce = n < cb + chunk ? n : cb + chunk;
    int64_t pos = cb;
    while (pos < ce) {
        int q = 0;
        int64_t qend = ce;
        if (sp.nsegs > 1) {
            q = seg_of(d_seg, sp.nsegs, pos);
            if (q + 1 < sp.nsegs) {
                const int64_t e = d_seg[q + 1];
                if (e > pos && e < ce) qend = e;
            }
        }
        if (MODE == kDenseDirect) {
            aggregate_range_dense<NA, true, PROBE>(sp, m, sel, pos, qend, q, g, max_groups, out_seg, status);
        } else {
            if (MODE == kDenseBlock)
                aggregate_range_dense<NA, false, PROBE>(sp, m, sel, pos, qend, q, g, max_groups, out_seg, status);
            else
                aggregate_range<NA>(sp, m, sel, pos, qend, q, g, max_groups, out_seg, status);
            flush_block_table(sp, m, q, g, max_groups, out_seg, status);
        }
        pos = qend;
    }
}

// Dense aggregation of the most common Partial shape (a join's output grouped by
// the gathered dimension attribute): one key column KT, SUM of one column VT and
// COUNT, no selection, a key range wide enough that one shared-memory replica of
// its slots serves every warp of the block without much collision, and a dense
// global result. Same contract as the dense block mode of groupby_kernel with
// far fewer instructions per row: each thread takes ITEMS consecutive rows with
// 16-byte vector loads, the SUM is held as 32-bit words (an atomic add on the low
// word returns the carry into the high word), COUNT is a plain 32-bit reduction,
// hot keys (lane 0's slot shared by >= kMajority lanes) are summed across the warp
// first, and each segment's slots are flushed into the dense global array.
// Rows whose key lies outside the range take the global hash path.
template <typename KT, typename VT, int ITEMS>
__global__ void __launch_bounds__(kThreads, 1)
groupby_sum_count_kernel(Spec sp, int32_t sum_slot, int32_t cnt_slot, const int64_t* __restrict__ d_n, int64_t ncap,
                         const int64_t* __restrict__ d_seg, GTable g, int64_t max_groups, int32_t* __restrict__ out_seg,
                         int32_t* status) {
    constexpr int T = kThreads * ITEMS;
    static_assert(ITEMS * sizeof(KT) % 16 == 0 && ITEMS * sizeof(VT) % 16 == 0, "whole 16-byte loads per thread");
    extern __shared__ __align__(16) uint32_t s_acc[];  // low words [D], high words [D], counts [D]
    const uint32_t D = sp.D;
    uint32_t* s_lo = s_acc;
    uint32_t* s_hi = s_acc + D;
    uint32_t* s_cnt = s_acc + 2 * static_cast<size_t>(D);
    const int tid = threadIdx.x, lane = tid & 31;
    for (uint32_t w = tid; w < 3 * D; w += kThreads) s_acc[w] = 0;
    __syncthreads();
    const KT* __restrict__ key = static_cast<const KT*>(sp.key_in[0]);
    const VT* __restrict__ val = static_cast<const VT*>(sp.a_in[sum_slot]);
    const int64_t lo = sp.lo[0];
    const int64_t n = actual_rows(d_n, ncap);
    // Each block owns a contiguous range of whole tiles and walks it segment by segment.
    const int64_t chunk = cdiv(cdiv(n, gridDim.x), T) * T;
    const int64_t cb = static_cast<int64_t>(blockIdx.x) * chunk;
    const int64_t ce = n < cb + chunk ? n : cb + chunk;
    int64_t pos = cb;
    while (pos < ce) {
        int q = 0;
        int64_t qend = ce;
        if (sp.nsegs > 1) {
            q = seg_of(d_seg, sp.nsegs, pos);
            if (q + 1 < sp.nsegs) {
                const int64_t e = d_seg[q + 1];
                if (e > pos && e < ce) qend = e;
            }
        }
        // Tiles aligned to T, rows outside [pos, qend) masked: a tile that straddles
        // a segment boundary is read once for each side.
        for (int64_t tb = pos / T * T; tb < qend; tb += T) {
            const int64_t r0 = tb + static_cast<int64_t>(tid) * ITEMS;
            KT k[ITEMS];
            VT v[ITEMS];
            if (r0 + ITEMS <= ncap) {
#pragma unroll
                for (int c = 0; c < ITEMS * static_cast<int>(sizeof(KT)) / 16; ++c)
                    reinterpret_cast<int4*>(k)[c] = reinterpret_cast<const int4*>(key + r0)[c];
#pragma unroll
                for (int c = 0; c < ITEMS * static_cast<int>(sizeof(VT)) / 16; ++c)
                    reinterpret_cast<int4*>(v)[c] = reinterpret_cast<const int4*>(val + r0)[c];
            } else {
#pragma unroll
                for (int i = 0; i < ITEMS; ++i) {
                    k[i] = r0 + i < ncap ? key[r0 + i] : KT(0);
                    v[i] = r0 + i < ncap ? val[r0 + i] : VT(0);
                }
            }
            uint32_t idx[ITEMS];
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const int64_t r = r0 + i;
                const uint64_t o = static_cast<uint64_t>(static_cast<int64_t>(k[i]) - lo);
                idx[i] = r < pos || r >= qend ? kIdxNone : (o < D ? static_cast<uint32_t>(o) : kIdxOutside);
            }
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const uint32_t c0 = __shfl_sync(FULL, idx[i], 0);
                const uint32_t mm = __ballot_sync(FULL, idx[i] == c0);
                uint64_t x = static_cast<uint64_t>(static_cast<int64_t>(v[i]));
                uint32_t cnt = 1;
                uint32_t d = idx[i];
                if (c0 < kIdxOutside && __popc(mm) >= kMajority) {  // warp-uniform
                    // Lane 0 (always in the group) applies the group's totals; the
                    // group's other lanes drop out; lanes outside it keep their row.
                    const bool in = (mm >> lane) & 1u;
                    const uint64_t total = warp_sum_u64(in ? x : 0);
                    if (lane == 0) {
                        x = total;
                        cnt = __popc(mm);
                    } else if (in) {
                        d = kIdxNone;
                    }
                }
                if (d < kIdxOutside) {
                    const uint32_t xl = static_cast<uint32_t>(x);
                    const uint32_t old = atomicAdd(&s_lo[d], xl);
                    const uint32_t h = static_cast<uint32_t>(x >> 32) + (old + xl < old ? 1u : 0u);
                    if (h) red_add_shared(&s_hi[d], h);
                    red_add_shared(&s_cnt[d], cnt);
                } else if (d == kIdxOutside) {
                    uint64_t full[2];
                    full[sum_slot] = x;
                    full[cnt_slot] = 1;
                    global_add(g, sp, compose(sp, static_cast<int64_t>(k[i]), 0, q), full, max_groups, out_seg, status);
                }
            }
        }
        // Segment q's slots into the dense global array, then cleared for the next.
        __syncthreads();
        const uint64_t ebase = static_cast<uint64_t>(q) * D;
        for (uint32_t d = tid; d < D; d += kThreads) {
            const uint32_t c = s_cnt[d];
            if (c) {
                red_add_global(&sp.dg_acc[sum_slot * sp.E + ebase + d],
                               (static_cast<unsigned long long>(s_hi[d]) << 32) | s_lo[d]);
                red_add_global(&sp.dg_acc[cnt_slot * sp.E + ebase + d], c);
                s_lo[d] = s_hi[d] = s_cnt[d] = 0;
            }
        }
        __syncthreads();
        pos = qend;
    }
}

template <typename KT, typename VT>
px_status launch_sum_count(const Spec& sp, int32_t sum_slot, int32_t cnt_slot, const int64_t* d_n, int64_t ncap,
                           const int64_t* d_seg, const GTable& g, int64_t max_groups, int32_t* out_seg,
                           int32_t* status, cudaStream_t st) {
    constexpr int ITEMS = 16 / sizeof(KT) > 16 / sizeof(VT) ? 16 / sizeof(KT) : 16 / sizeof(VT);
    auto kernel = groupby_sum_count_kernel<KT, VT, ITEMS>;
    const size_t smem = 12 * static_cast<size_t>(sp.D);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    // A block flushes its D slots at every segment end: give each at least 4 D rows.
    const int64_t grid = std::max<int64_t>(
        1, std::min<int64_t>(cdiv(ncap, std::max<int64_t>(kThreads * ITEMS, 4 * static_cast<int64_t>(sp.D))),
                             sm_count()));
    kernel<<<static_cast<unsigned>(grid), kThreads, smem, st>>>(sp, sum_slot, cnt_slot, d_n, ncap, d_seg, g,
                                                              max_groups, out_seg, status);
    note_launch();
    return check_launch("px_groupby_agg sum-count");
}

// px_join_probe_agg's SUM + COUNT shape with the lean kernel's accumulation:
// every position's key is looked up in its segment of the join table (one sector:
// keys, build rows and the group column copied beside them; a walk on for the
// keys displaced past their home bucket), its group's dense slot comes from the
// copied value (else from a gather of the group column), and its amount is added
// to the block's slot as in groupby_sum_count_kernel. The joined rows are never
// written. Two positions per thread (one 16-byte load of their keys).
template <typename VT>
__global__ void __launch_bounds__(kThreads, 1)
groupby_probe_sum_count_kernel(Spec sp, int32_t sum_slot, int32_t cnt_slot, const int64_t* __restrict__ d_n,
                               int64_t ncap, const int64_t* __restrict__ d_seg, GTable g, int64_t max_groups,
                               int32_t* __restrict__ out_seg, int32_t* status) {
    constexpr int ITEMS = 2;
    constexpr int T = kThreads * ITEMS;
    extern __shared__ __align__(16) uint32_t s_acc[];  // low words [D], high words [D], counts [D]
    const uint32_t D = sp.D;
    uint32_t* s_lo = s_acc;
    uint32_t* s_hi = s_acc + D;
    uint32_t* s_cnt = s_acc + 2 * static_cast<size_t>(D);
    const int tid = threadIdx.x, lane = tid & 31;
    for (uint32_t w = tid; w < 3 * D; w += kThreads) s_acc[w] = 0;
    __syncthreads();
    const TableHeader* h = sp.probe_t.hdr;
    const int S = sp.nsegs > 0 ? sp.nsegs : 1;
    if (h->magic != kMagic || h->nsegs != S || h->unique == 0 || h->nbuild > sp.nbuild) {  // unusable table
        if (blockIdx.x == 0 && tid == 0)
            set_status(status, h->magic == kMagic && h->unique == 0 ? PX_ERR_UNSUPPORTED : PX_ERR_INVALID);
        return;
    }
    const bool group_in_table = h->pay_src == sp.group_col && h->pay_w == sp.group_w;
    const int64_t* __restrict__ fk = sp.probe_fk;
    const VT* __restrict__ val = static_cast<const VT*>(sp.a_in[sum_slot]);
    const int64_t lo = sp.lo[0];
    const int64_t n = actual_rows(d_n, ncap);
    const int64_t chunk = cdiv(cdiv(n, gridDim.x), T) * T;
    const int64_t cb = static_cast<int64_t>(blockIdx.x) * chunk;
    const int64_t ce = n < cb + chunk ? n : cb + chunk;
    // The keys and amounts of the next tile to visit are loaded while the current
    // tile's buckets are in flight (one memory round trip per tile, not two).
    auto load_tile = [&](int64_t tb, int64_t* k, VT* v) {
        const int64_t r0 = tb + static_cast<int64_t>(tid) * ITEMS;
        if (r0 + ITEMS <= ncap) {
            const longlong2 k2 = *reinterpret_cast<const longlong2*>(fk + r0);
            k[0] = k2.x;
            k[1] = k2.y;
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) v[i] = val[r0 + i];
        } else {
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                k[i] = r0 + i < ncap ? fk[r0 + i] : kEmpty;
                v[i] = r0 + i < ncap ? val[r0 + i] : VT(0);
            }
        }
    };
    int64_t kn[ITEMS];
    VT vn[ITEMS];
    if (cb < ce) load_tile(cb, kn, vn);
    int64_t pos = cb;
    while (pos < ce) {
        int q = 0;
        int64_t qend = ce;
        if (sp.nsegs > 1) {
            q = seg_of(d_seg, sp.nsegs, pos);
            if (q + 1 < sp.nsegs) {
                const int64_t e = d_seg[q + 1];
                if (e > pos && e < ce) qend = e;
            }
        }
        const SegGeom geo = seg_geom(sp.probe_t, q);
        const Bucket* const segb = sp.probe_t.bk + geo.b0;
        for (int64_t tb = pos / T * T; tb < qend; tb += T) {
            const int64_t r0 = tb + static_cast<int64_t>(tid) * ITEMS;
            int64_t k[ITEMS];
            VT v[ITEMS];
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                k[i] = kn[i];
                v[i] = vn[i];
            }
            bool live[ITEMS];
            uint32_t hb[ITEMS];
            BucketRegs bv[ITEMS];
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const int64_t r = r0 + i;
                live[i] = r >= pos && r < qend && k[i] != kEmpty;
                hb[i] = home_bucket(static_cast<uint64_t>(k[i]), geo.nb);
                bv[i] = load_bucket(segb + hb[i]);  // hb < nb: inside the segment
            }
            // next visit: this segment's next tile, or the tile where the next segment starts
            const int64_t nxt = tb + T < qend ? tb + T : (qend < ce ? qend / T * T : -1);
            if (nxt >= 0) load_tile(nxt, kn, vn);
            uint32_t idx[ITEMS];
            int64_t gk[ITEMS];
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                idx[i] = kIdxNone;
                gk[i] = 0;
                if (!live[i]) continue;
                bool end;
                int l = bucket_find(bv[i], k[i], &end);
                if (l < 0 && !end) l = walk_find(segb, geo.nb, hb[i], k[i], &bv[i]);
                if (l < 0) continue;  // no match: no group
                gk[i] = group_in_table ? static_cast<int64_t>(bucket_pay(bv[i], l))
                                       : load_int(sp.group_col, sp.group_w, bucket_row(bv[i], l));
                const uint64_t o = static_cast<uint64_t>(gk[i] - lo);
                idx[i] = o < D ? static_cast<uint32_t>(o) : kIdxOutside;
            }
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const uint32_t c0 = __shfl_sync(FULL, idx[i], 0);
                const uint32_t mm = __ballot_sync(FULL, idx[i] == c0);
                uint64_t x = static_cast<uint64_t>(static_cast<int64_t>(v[i]));
                uint32_t cnt = 1;
                uint32_t d = idx[i];
                if (c0 < kIdxOutside && __popc(mm) >= kMajority) {  // warp-uniform
                    // Lane 0 (always in the group) applies the group's totals; the
                    // group's other lanes drop out; lanes outside it keep their row.
                    const bool in = (mm >> lane) & 1u;
                    const uint64_t total = warp_sum_u64(in ? x : 0);
                    if (lane == 0) {
                        x = total;
                        cnt = __popc(mm);
                    } else if (in) {
                        d = kIdxNone;
                    }
                }
                if (d < kIdxOutside) {
                    const uint32_t xl = static_cast<uint32_t>(x);
                    const uint32_t old = atomicAdd(&s_lo[d], xl);
                    const uint32_t hi = static_cast<uint32_t>(x >> 32) + (old + xl < old ? 1u : 0u);
                    if (hi) red_add_shared(&s_hi[d], hi);
                    red_add_shared(&s_cnt[d], cnt);
                } else if (d == kIdxOutside) {
                    uint64_t full[2];
                    full[sum_slot] = x;
                    full[cnt_slot] = 1;
                    global_add(g, sp, compose(sp, gk[i], 0, q), full, max_groups, out_seg, status);
                }
            }
        }
        // Segment q's slots into the dense global array, then cleared for the next.
        __syncthreads();
        const uint64_t ebase = static_cast<uint64_t>(q) * D;
        for (uint32_t d = tid; d < D; d += kThreads) {
            const uint32_t c = s_cnt[d];
            if (c) {
                red_add_global(&sp.dg_acc[sum_slot * sp.E + ebase + d],
                               (static_cast<unsigned long long>(s_hi[d]) << 32) | s_lo[d]);
                red_add_global(&sp.dg_acc[cnt_slot * sp.E + ebase + d], c);
                s_lo[d] = s_hi[d] = s_cnt[d] = 0;
            }
        }
        __syncthreads();
        pos = qend;
    }
}

template <typename VT>
px_status launch_probe_sum_count(const Spec& sp, int32_t sum_slot, int32_t cnt_slot, const int64_t* d_n, int64_t ncap,
                                 const int64_t* d_seg, const GTable& g, int64_t max_groups, int32_t* out_seg,
                                 int32_t* status, cudaStream_t st) {
    auto kernel = groupby_probe_sum_count_kernel<VT>;
    const size_t smem = 12 * static_cast<size_t>(sp.D);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    const int64_t grid = std::max<int64_t>(
        1, std::min<int64_t>(cdiv(ncap, std::max<int64_t>(kThreads * 2, 4 * static_cast<int64_t>(sp.D))), sm_count()));
    kernel<<<static_cast<unsigned>(grid), kThreads, smem, st>>>(sp, sum_slot, cnt_slot, d_n, ncap, d_seg, g,
                                                              max_groups, out_seg, status);
    note_launch();
    return check_launch("px_join_probe_agg sum-count");
}

constexpr int kEmitThreads = 256;
constexpr int kEmitItems = 8;
constexpr int kEmitTile = kEmitThreads * kEmitItems;
constexpr int kEmitWarps = kEmitThreads / 32;

// Writes the occupied entries of the dense global array as output groups, in
// (segment, key) order, after the groups the hash path claimed (rows whose keys
// fell outside the key range). Single pass with a bounded look-back.
__global__ void __launch_bounds__(kEmitThreads)
dense_emit_kernel(Spec sp, const unsigned long long* __restrict__ ngroups_hash, int64_t max_groups,
                  int32_t* __restrict__ out_seg, int64_t* __restrict__ d_ngroups, ScanScratch scan, int32_t* status,
                  int64_t ntiles) {
    __shared__ int64_t s_tile;
    __shared__ int64_t s_excl;
    __shared__ int32_t s_warp[kEmitWarps];
    const int64_t tile = next_tile(scan.counter, &s_tile);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = tile * kEmitTile + warp * (32 * kEmitItems);
    const int64_t E = static_cast<int64_t>(sp.E);
    const int64_t first = static_cast<int64_t>(*ngroups_hash);
    uint32_t mask[kEmitItems];
    int32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < kEmitItems; ++i) {
        const int64_t e = base + i * 32 + lane;
        bool occ = false;
        if (e < E)
            occ = sp.count_agg >= 0 ? sp.dg_acc[sp.count_agg * E + e] != 0 : sp.dg_occ[e] != 0;
        mask[i] = __ballot_sync(FULL, occ);
        cnt += __popc(mask[i]);
    }
    if (lane == 0) s_warp[warp] = cnt;
    __syncthreads();
    if (warp == 0) {
        const int32_t w = lane < kEmitWarps ? s_warp[lane] : 0;
        const int32_t incl = warp_incl_scan(w);
        const int32_t total = __shfl_sync(FULL, incl, 31);
        if (lane < kEmitWarps) s_warp[lane] = incl - w;
        const int64_t excl = lookback(scan.states, tile, total, status);
        if (lane == 0) {
            s_excl = excl;
            if (tile == ntiles - 1) {
                *d_ngroups = first + excl + total;
                if (first + excl + total > max_groups) set_status(status, PX_ERR_CAPACITY);
            }
        }
    }
    __syncthreads();
    int64_t pos = first + s_excl + s_warp[warp];
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kEmitItems; ++i) {
        if (mask[i] & (1u << lane)) {
            const int64_t e = base + i * 32 + lane;
            const int64_t p = pos + __popc(mask[i] & lt);
            if (p < max_groups) {
                const uint64_t q = static_cast<uint64_t>(e) / sp.D;
                const uint64_t d = static_cast<uint64_t>(e) % sp.D;
                store_int(sp.key_out[0], sp.key_w[0], p, sp.lo[0] + static_cast<int64_t>(d / sp.span[1]));
                if (sp.nkeys > 1)
                    store_int(sp.key_out[1], sp.key_w[1], p, sp.lo[1] + static_cast<int64_t>(d % sp.span[1]));
                if (out_seg) out_seg[p] = static_cast<int32_t>(q);
                for (int a = 0; a < sp.naggs; ++a) sp.agg_out[a][p] = static_cast<int64_t>(sp.dg_acc[a * E + e]);
            }
        }
        pos += __popc(mask[i]);
    }
}

uint32_t gtable_slots(int64_t max_groups) {
    uint64_t G = 1024;
    while (G < 2 * static_cast<uint64_t>(max_groups)) G <<= 1;
    return static_cast<uint32_t>(G);
}

uint32_t hash_slots(int naggs) {
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

template <int NA, int MODE, bool PROBE = false>
px_status launch_mode(const Spec& sp, size_t smem, const int32_t* sel, const int64_t* d_n, int64_t ncap,
                      const int64_t* d_seg, const GTable& g, int64_t max_groups, int32_t* out_seg, int32_t* status,
                      uint32_t hslots, cudaStream_t st) {
    auto kernel = groupby_kernel<NA, MODE, PROBE>;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem);
    // A dense block flushes its D slots into the global result at every segment end,
    // so each block gets at least 4 D rows: fewer blocks for small inputs, whose
    // flushes would otherwise pile same-address atomics onto the global array.
    const int64_t min_rows =
        MODE == kDenseBlock ? std::max<int64_t>(kTile, 4 * static_cast<int64_t>(sp.D)) : kTile;
    const int64_t grid = std::max<int64_t>(
        1, std::min<int64_t>(cdiv(ncap, min_rows), static_cast<int64_t>(num_sms()) * std::max(1, per_sm)));
    kernel<<<static_cast<unsigned>(grid), kThreads, smem, st>>>(sp, sel, d_n, ncap, d_seg, g, max_groups, out_seg,
                                                                status, hslots);
    note_launch();
    return check_launch("px_groupby_agg");
}

// Fused probe: dense modes only (the caller guarantees sp.dense).
template <int NA>
px_status launch_probe(const Spec& sp, size_t smem, const int32_t* sel, const int64_t* d_n, int64_t ncap,
                       const int64_t* d_seg, const GTable& g, int64_t max_groups, int32_t* out_seg, int32_t* status,
                       uint32_t hslots, cudaStream_t st) {
    if (sp.direct)
        return launch_mode<NA, kDenseDirect, true>(sp, smem, sel, d_n, ncap, d_seg, g, max_groups, out_seg, status,
                                                   hslots, st);
    return launch_mode<NA, kDenseBlock, true>(sp, smem, sel, d_n, ncap, d_seg, g, max_groups, out_seg, status, hslots,
                                              st);
}

template <int NA>
px_status launch(const Spec& sp, size_t smem, const int32_t* sel, const int64_t* d_n, int64_t ncap,
                 const int64_t* d_seg, const GTable& g, int64_t max_groups, int32_t* out_seg, int32_t* status,
                 uint32_t hslots, cudaStream_t st) {
    if (sp.probe_fk)
        return launch_probe<NA>(sp, smem, sel, d_n, ncap, d_seg, g, max_groups, out_seg, status, hslots, st);
    if (sp.direct)
        return launch_mode<NA, kDenseDirect>(sp, smem, sel, d_n, ncap, d_seg, g, max_groups, out_seg, status, hslots,
                                             st);
    if (sp.dense)
        return launch_mode<NA, kDenseBlock>(sp, smem, sel, d_n, ncap, d_seg, g, max_groups, out_seg, status, hslots,
                                            st);
    return launch_mode<NA, kHashed>(sp, smem, sel, d_n, ncap, d_seg, g, max_groups, out_seg, status, hslots, st);
}

}  // namespace
}  // namespace px

using namespace px;

extern "C" {

// Workspace: [header][group counter][hash table: state, key, gidx (G slots)]
// [dense global: acc (PX_MAX_AGGS x max_groups), occupancy flags (1 byte each)][emit scan scratch].
struct WsLayout {
    size_t counter, state, key, gidx, dg_acc, dg_occ, emit_scan, total;
};

WsLayout ws_layout(int64_t max_groups) {
    if (max_groups < 1) max_groups = 1;
    const size_t G = gtable_slots(max_groups);
    const size_t M = static_cast<size_t>(max_groups);
    WsLayout L;
    L.counter = kWsScratch;
    L.state = L.counter + 256;
    L.key = L.state + align_up(4 * G, 256);
    L.gidx = L.key + align_up(8 * G, 256);
    L.dg_acc = L.gidx + align_up(4 * G, 256);
    L.dg_occ = L.dg_acc + align_up(8 * PX_MAX_AGGS * M, 256);
    L.emit_scan = L.dg_occ + align_up(M, 256);
    L.total = L.emit_scan + scan_scratch_bytes(cdiv(static_cast<int64_t>(M), kEmitTile));
    return L;
}

size_t px_groupby_ws_bytes(int64_t nrows, int64_t max_groups) {
    (void)nrows;
    return ws_layout(max_groups).total;
}

// The fused join probe of px_join_probe_agg: the key of a position is the group
// column at the build row its fk matches in the table.
struct ProbeSrc {
    const void* table;
    int32_t fk_col;
    const px_col* group;
    int64_t nbuild;
};

static px_status groupby_impl(const px_batch* in, const int32_t* key_cols, int32_t nkeys, const px_agg* aggs,
                              int32_t naggs, const int32_t* d_sel, const int64_t* d_nsel, const int64_t* d_seg,
                              int32_t nsegs, const px_key_range* range, int64_t max_groups, const px_batch* out,
                              int32_t* d_out_seg, int64_t* d_ngroups, int32_t flags, void* d_ws, size_t ws_bytes,
                              void* stream, const ProbeSrc* probe = nullptr) {
    set_error("");
    if (flags & ~(PX_AGG_ACCUMULATE | PX_AGG_STREAM))
        return fail(PX_ERR_INVALID, "px_groupby_agg_stream: unknown flags 0x%x", flags);
    const bool accumulate = (flags & PX_AGG_ACCUMULATE) != 0;
    const bool streaming = accumulate || (flags & PX_AGG_STREAM) != 0;
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
    Spec sp = {};
    sp.nkeys = nkeys;
    sp.keybits = 0;
    for (int k = 0; k < nkeys; ++k) {
        if (!probe && (key_cols[k] < 0 || key_cols[k] >= in->ncols))
            return fail(PX_ERR_INVALID, "px_groupby_agg: key column %d out of range", key_cols[k]);
        const px_col& c = probe ? *probe->group : in->cols[key_cols[k]];
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
    sp.count_agg = -1;
    for (int a = 0; a < naggs; ++a) {
        const px_agg& ag = aggs[a];
        if (ag.op != PX_COUNT && ag.op != PX_SUM && ag.op != PX_SUM_MUL)
            return fail(PX_ERR_INVALID, "px_groupby_agg: aggregate %d has unknown op %d", a, ag.op);
        sp.op[a] = ag.op;
        sp.a_w[a] = sp.b_w[a] = 8;
        sp.a_in[a] = sp.b_in[a] = nullptr;
        if (ag.op == PX_COUNT && sp.count_agg < 0) sp.count_agg = a;
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

    // Dense modes when the key statistic makes the key space small enough: rows go
    // straight into a dense global array when every (segment, key) entry fits
    // max_groups and there are too few rows to give each SM a block that amortises
    // clearing and flushing D block slots; else dense block arrays when they fit
    // shared memory; else hashing.
    size_t smem = 0;
    sp.dense = 0;
    sp.direct = 0;
    sp.reps = 1;
    sp.span[0] = sp.span[1] = 1;
    if (range) {
        bool ok = true;
        uint64_t D = 1;
        for (int k = 0; k < nkeys && ok; ++k) {
            if (range->hi[k] < range->lo[k]) {
                ok = false;
                break;
            }
            const uint64_t span = static_cast<uint64_t>(range->hi[k]) - static_cast<uint64_t>(range->lo[k]) + 1;
            if (span == 0 || span > (1ull << 24)) ok = false;
            sp.lo[k] = range->lo[k];
            sp.span[k] = span;
            D *= span;
        }
        if (ok && D <= (1ull << 24)) {
            sp.n64 = sp.n32 = 0;
            for (int a = 0; a < naggs; ++a) {
                sp.kind[a] = sp.op[a] == PX_COUNT ? 1 : 0;
                sp.slot[a] = sp.kind[a] ? sp.n32++ : sp.n64++;
            }
            size_t per_rep = static_cast<size_t>(sp.n64) * D * 8 + static_cast<size_t>(sp.n32) * D * 4 +
                             (sp.count_agg < 0 ? (D + 31) / 32 * 4 : 0);
            per_rep = align_up(per_rep, 8);
            const uint64_t E = static_cast<uint64_t>(nsegs > 0 ? nsegs : 1) * D;
            // A stream of calls keeps its groups in one place: the choice then depends
            // on the statistic and max_groups only, never on the row count.
            const bool few_rows =
                streaming ? per_rep > kSmemBudget
                          : cdiv(in->nrows, std::max<int64_t>(kTile, 4 * static_cast<int64_t>(D))) < num_sms();
            if (E <= static_cast<uint64_t>(max_groups) && few_rows) {
                sp.dense = 1;
                sp.direct = 1;
                sp.D = static_cast<uint32_t>(D);
            } else if (per_rep > 0 && per_rep <= kSmemBudget) {
                sp.dense = 1;
                sp.D = static_cast<uint32_t>(D);
                // One replica per thread when they fit (plain adds, no contention),
                // with an odd number of 8-byte words per replica to spread the banks;
                // else up to one per warp.
                const size_t priv = (per_rep / 8) % 2 == 0 ? per_rep + 8 : per_rep;
                if (priv * kThreads <= kSmemBudget) {
                    sp.reps = kThreads;
                    sp.rep_bytes = static_cast<uint32_t>(priv);
                } else {
                    while (sp.reps * 2 <= kWarps && per_rep * sp.reps * 2 <= kSmemBudget) sp.reps *= 2;
                    sp.rep_bytes = static_cast<uint32_t>(per_rep);
                }
                smem = static_cast<size_t>(sp.rep_bytes) * sp.reps;
            }
        }
    }
    if (probe) {
        if (!sp.dense)
            return fail(PX_ERR_UNSUPPORTED,
                        "px_join_probe_agg: needs a group key range small enough for dense aggregation");
        sp.probe_fk = static_cast<const int64_t*>(in->cols[probe->fk_col].data);
        sp.probe_t = table_view(const_cast<void*>(probe->table), nsegs > 0 ? nsegs : 1);
        sp.group_col = probe->group->data;
        sp.group_w = probe->group->type;
        sp.nbuild = probe->nbuild;
    }
    const uint32_t hslots = hash_slots(naggs);
    if (!sp.dense) smem = static_cast<size_t>(hslots) * (12 + 8 * static_cast<size_t>(naggs));

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t G = gtable_slots(max_groups);
    const WsLayout L = ws_layout(max_groups);
    char* ws = static_cast<char*>(d_ws);
    GTable g;
    g.ngroups = reinterpret_cast<unsigned long long*>(ws + L.counter);
    g.state = reinterpret_cast<uint32_t*>(ws + L.state);
    g.key = reinterpret_cast<unsigned long long*>(ws + L.key);
    g.gidx = reinterpret_cast<int32_t*>(ws + L.gidx);
    g.mask = G - 1;
    if (!accumulate) cudaMemsetAsync(ws + L.counter, 0, 256 + 4ull * G, st);
    // Dense global result when the whole (segment, key) space fits max_groups.
    sp.dglobal = 0;
    if (sp.dense) {
        const uint64_t E = static_cast<uint64_t>(nsegs > 0 ? nsegs : 1) * sp.D;
        if (E <= static_cast<uint64_t>(max_groups)) {
            sp.dglobal = 1;
            sp.E = E;
            sp.dg_acc = reinterpret_cast<unsigned long long*>(ws + L.dg_acc);
            sp.dg_occ = reinterpret_cast<uint8_t*>(ws + L.dg_occ);
            if (!accumulate) {
                cudaMemsetAsync(sp.dg_acc, 0, 8ull * naggs * E, st);
                if (sp.count_agg < 0) cudaMemsetAsync(sp.dg_occ, 0, E, st);
            }
        }
    }
    const int64_t ncap = in->nrows;
    int32_t* status = &static_cast<WsHeader*>(d_ws)->status;
    // The lean kernel of the SUM + COUNT shape (see groupby_sum_count_kernel):
    // one key of 4 or 8 bytes, a dense block mode with one replica of a dense
    // global result, no selection, not fused with a probe.
    int32_t sum_slot = -1, cnt_slot = -1;
    if (naggs == 2)
        for (int a = 0; a < 2; ++a) {
            if (sp.op[a] == PX_COUNT) cnt_slot = a;
            else if (sp.op[a] == PX_SUM && (sp.a_w[a] == 8 || sp.a_w[a] == 4)) sum_slot = a;
        }
    const bool sum_count = ncap > 0 && !probe && sp.dense && !sp.direct && sp.dglobal && sp.reps == 1 &&
                           d_sel == nullptr && nkeys == 1 && (sp.key_w[0] == 4 || sp.key_w[0] == 8) &&
                           sum_slot >= 0 && cnt_slot >= 0 && 12 * static_cast<size_t>(sp.D) <= kSmemBudget;
    // The same shape fed by the join probe, with the rows' keys looked up in the table.
    const bool probe_sum_count = ncap > 0 && probe && sp.dense && !sp.direct && sp.dglobal && sp.reps == 1 &&
                                 d_sel == nullptr && nkeys == 1 && sum_slot >= 0 && cnt_slot >= 0 &&
                                 12 * static_cast<size_t>(sp.D) <= kSmemBudget;
    if (probe_sum_count) {
        const int64_t* d_n = in->d_nrows;
        s = sp.a_w[sum_slot] == 8
                ? launch_probe_sum_count<int64_t>(sp, sum_slot, cnt_slot, d_n, ncap, d_seg, g, max_groups, d_out_seg,
                                                  status, st)
                : launch_probe_sum_count<int32_t>(sp, sum_slot, cnt_slot, d_n, ncap, d_seg, g, max_groups, d_out_seg,
                                                  status, st);
        if (s != PX_OK) return s;
    } else if (sum_count) {
        const int64_t* d_n = in->d_nrows;
        if (sp.key_w[0] == 4 && sp.a_w[sum_slot] == 8)
            s = launch_sum_count<int32_t, int64_t>(sp, sum_slot, cnt_slot, d_n, ncap, d_seg, g, max_groups, d_out_seg,
                                                   status, st);
        else if (sp.key_w[0] == 4)
            s = launch_sum_count<int32_t, int32_t>(sp, sum_slot, cnt_slot, d_n, ncap, d_seg, g, max_groups, d_out_seg,
                                                   status, st);
        else if (sp.a_w[sum_slot] == 8)
            s = launch_sum_count<int64_t, int64_t>(sp, sum_slot, cnt_slot, d_n, ncap, d_seg, g, max_groups, d_out_seg,
                                                   status, st);
        else
            s = launch_sum_count<int64_t, int32_t>(sp, sum_slot, cnt_slot, d_n, ncap, d_seg, g, max_groups, d_out_seg,
                                                   status, st);
        if (s != PX_OK) return s;
    } else if (ncap > 0) {
        const int64_t* d_n = d_sel ? d_nsel : in->d_nrows;
        switch (naggs) {
            case 0: s = launch<0>(sp, smem, d_sel, d_n, ncap, d_seg, g, max_groups, d_out_seg, status, hslots, st); break;
            case 1: s = launch<1>(sp, smem, d_sel, d_n, ncap, d_seg, g, max_groups, d_out_seg, status, hslots, st); break;
            case 2: s = launch<2>(sp, smem, d_sel, d_n, ncap, d_seg, g, max_groups, d_out_seg, status, hslots, st); break;
            case 3: s = launch<3>(sp, smem, d_sel, d_n, ncap, d_seg, g, max_groups, d_out_seg, status, hslots, st); break;
            case 4: s = launch<4>(sp, smem, d_sel, d_n, ncap, d_seg, g, max_groups, d_out_seg, status, hslots, st); break;
            default:
                s = launch<PX_MAX_AGGS>(sp, smem, d_sel, d_n, ncap, d_seg, g, max_groups, d_out_seg, status, hslots,
                                        st);
                break;
        }
        if (s != PX_OK) return s;
    }
    if (sp.dglobal) {
        const int64_t ntiles = cdiv(static_cast<int64_t>(sp.E), kEmitTile);
        cudaMemsetAsync(ws + L.emit_scan, 0, scan_scratch_bytes(ntiles), st);
        dense_emit_kernel<<<static_cast<unsigned>(ntiles), kEmitThreads, 0, st>>>(
            sp, g.ngroups, max_groups, d_out_seg, d_ngroups, scan_scratch(ws + L.emit_scan), status, ntiles);
        note_launch();
        return check_launch("px_groupby_agg emit");
    }
    cudaMemcpyAsync(d_ngroups, g.ngroups, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    return check_launch("px_groupby_agg count");
}

px_status px_groupby_agg(const px_batch* in, const int32_t* key_cols, int32_t nkeys, const px_agg* aggs,
                         int32_t naggs, const int32_t* d_sel, const int64_t* d_nsel, const int64_t* d_seg,
                         int32_t nsegs, const px_key_range* range, int64_t max_groups, const px_batch* out,
                         int32_t* d_out_seg, int64_t* d_ngroups, void* d_ws, size_t ws_bytes, void* stream) {
    CallRange nvtx_range("px_groupby_agg");
    return groupby_impl(in, key_cols, nkeys, aggs, naggs, d_sel, d_nsel, d_seg, nsegs, range, max_groups, out,
                        d_out_seg, d_ngroups, 0, d_ws, ws_bytes, stream);
}

px_status px_groupby_agg_stream(const px_batch* in, const int32_t* key_cols, int32_t nkeys, const px_agg* aggs,
                                int32_t naggs, const int32_t* d_sel, const int64_t* d_nsel, const int64_t* d_seg,
                                int32_t nsegs, const px_key_range* range, int64_t max_groups, const px_batch* out,
                                int32_t* d_out_seg, int64_t* d_ngroups, int32_t flags, void* d_ws, size_t ws_bytes,
                                void* stream) {
    CallRange nvtx_range("px_groupby_agg_stream");
    return groupby_impl(in, key_cols, nkeys, aggs, naggs, d_sel, d_nsel, d_seg, nsegs, range, max_groups, out,
                        d_out_seg, d_ngroups, flags, d_ws, ws_bytes, stream);
}

size_t px_join_probe_agg_ws_bytes(int64_t nprobe, int64_t max_groups) { return px_groupby_ws_bytes(nprobe, max_groups); }

px_status px_join_probe_agg(const void* d_table, const px_batch* probe, int32_t fk_col, const int32_t* d_sel,
                            const int64_t* d_nsel, const int64_t* d_seg, int32_t nsegs, const px_col* group,
                            int64_t nbuild, int64_t group_lo, int64_t group_hi, const px_agg* aggs, int32_t naggs,
                            int64_t max_groups, const px_batch* out, int32_t* d_out_seg, int64_t* d_ngroups,
                            void* d_ws, size_t ws_bytes, void* stream) {
    CallRange nvtx_range("px_join_probe_agg");
    set_error("");
    px_status s = check_batch(probe, "px_join_probe_agg probe");
    if (s != PX_OK) return s;
    if (!d_table || !aligned16(d_table)) return fail(PX_ERR_INVALID, "px_join_probe_agg: null or misaligned table");
    if (fk_col < 0 || fk_col >= probe->ncols || probe->cols[fk_col].type != PX_I64)
        return fail(PX_ERR_INVALID, "px_join_probe_agg: fk_col must name a PX_I64 probe column");
    if (!group || nbuild < 0) return fail(PX_ERR_INVALID, "px_join_probe_agg: group column");
    s = check_col(group, "px_join_probe_agg group", nbuild == 0);
    if (s != PX_OK) return s;
    if (group_hi < group_lo) return fail(PX_ERR_INVALID, "px_join_probe_agg: empty group range");
    px_key_range r = {};
    r.lo[0] = group_lo;
    r.hi[0] = group_hi;
    const int32_t key0 = 0;
    const ProbeSrc ps = {d_table, fk_col, group, nbuild};
    return groupby_impl(probe, &key0, 1, aggs, naggs, d_sel, d_nsel, d_seg, nsegs, &r, max_groups, out, d_out_seg,
                        d_ngroups, 0, d_ws, ws_bytes, stream, &ps);
}

}  // extern "C"
