// Join hash table layout shared by the join (px_join.cu), the probe-fed group-by
// (px_groupby.cu) and the fused fragment pipelines (px_fragments.cu). The table is
// caller memory:
//   [0, 64)            header: magic, nsegs, unique flag, build rows, embedded
//                      payload column (source address and width, 0 for none)
//   [64, 64 + A)       copy of the build segment offsets (nsegs + 1 int64)
//   [64 + A + p, ...)  buckets of 32 bytes (one DRAM/L2 sector): 2 int64 keys,
//                      their 2 int32 build rows and 2 int32 payload values; p < 32
//                      pads the first bucket to a 32-byte address (the caller's
//                      table is only 16-byte aligned), so one 32-byte vector load
//                      reads a whole bucket
// Segment q of n_q rows owns buckets [b_q, b_{q+1}) with b_q = seg[q] + q, i.e.
// n_q + 1 buckets = 2 n_q + 2 slots (load factor < 1/2). Slots are numbered
// 2 * bucket + lane; linear probing over slots starts at the first slot of the
// key's home bucket. Empty slots hold the key INT64_MIN. A lookup reads one sector
// for its key, build row and payload; about one key in eight sits past its home
// bucket at this load factor and reads the next bucket too.
#pragma once

#include "px_common.cuh"

namespace px {

constexpr int64_t kEmpty = INT64_MIN;
constexpr int64_t kMagic = 0x707874626c763033ll;  // "pxtblv03"
constexpr int kSlots = 2;                         // slots per bucket

struct TableHeader {
    int64_t magic;
    int32_t nsegs;   // >= 1
    int32_t unique;
    int64_t nbuild;        // build rows inserted
    const void* pay_src;   // build column copied into the buckets' payload slots
    int32_t pay_w;         // its width in bytes (1 or 4), 0 when there is none
    int32_t pad0;
    int64_t reserved[3];
};
static_assert(sizeof(TableHeader) == 64, "header is one 64-byte block");

struct Bucket {
    int64_t key[kSlots];
    int32_t row[kSlots];
    int32_t pay[kSlots];
};
static_assert(sizeof(Bucket) == 32, "bucket is one 32-byte sector");

inline size_t seg_area_bytes(int32_t S) { return align_up(static_cast<size_t>(S + 1) * 8, 64); }
__host__ __device__ inline int64_t table_buckets(int64_t n, int32_t S) { return n + S; }

struct TableView {
    TableHeader* hdr;
    int64_t* seg;
    Bucket* bk;
};

inline TableView table_view(void* d_table, int32_t S) {
    TableView t;
    char* b = static_cast<char*>(d_table);
    t.hdr = reinterpret_cast<TableHeader*>(b);
    t.seg = reinterpret_cast<int64_t*>(b + 64);
    const uintptr_t bk = reinterpret_cast<uintptr_t>(b + 64 + seg_area_bytes(S));
    t.bk = reinterpret_cast<Bucket*>((bk + 31) & ~static_cast<uintptr_t>(31));
    return t;
}

// Buckets of segment q: [b0, b0 + nb).
struct SegGeom {
    int64_t b0;
    uint32_t nb;
};
__device__ __forceinline__ SegGeom seg_geom(const TableView& t, int q) {
    const int64_t s0 = t.seg[q], s1 = t.seg[q + 1];
    SegGeom g;
    g.b0 = s0 + q;
    g.nb = static_cast<uint32_t>(s1 - s0 + 1);
    return g;
}

__device__ __forceinline__ uint32_t home_bucket(uint64_t key, uint32_t nb) { return slot_of(fmix64(key), nb); }

// One bucket in registers, read with a single 32-byte load.
struct BucketRegs {
    int64_t k0, k1;
    int32_t r0, r1, p0, p1;
};
__device__ __forceinline__ BucketRegs load_bucket(const Bucket* b) {
    const longlong4_32a v = *reinterpret_cast<const longlong4_32a*>(b);
    BucketRegs r;
    r.k0 = v.x;
    r.k1 = v.y;
    r.r0 = static_cast<int32_t>(static_cast<uint64_t>(v.z));
    r.r1 = static_cast<int32_t>(static_cast<uint64_t>(v.z) >> 32);
    r.p0 = static_cast<int32_t>(static_cast<uint64_t>(v.w));
    r.p1 = static_cast<int32_t>(static_cast<uint64_t>(v.w) >> 32);
    return r;
}

// Looks `key` up in one bucket: the lane of the match, or -1 with *end set when an
// empty slot ends the probe sequence in this bucket. Occupied slots form a prefix
// of every probe sequence and of every bucket (inserts take the first empty slot
// and slots never empty again), so the bucket's last slot tells whether it is full.
// A key equal to kEmpty must be excluded by the caller.
__device__ __forceinline__ int bucket_find(const BucketRegs& b, int64_t key, bool* end) {
    const int l = b.k0 == key ? 0 : (b.k1 == key ? 1 : -1);
    *end = l < 0 && b.k1 == kEmpty;
    return l;
}
__device__ __forceinline__ int32_t bucket_row(const BucketRegs& b, int l) { return l == 0 ? b.r0 : b.r1; }
__device__ __forceinline__ int32_t bucket_pay(const BucketRegs& b, int l) { return l == 0 ? b.p0 : b.p1; }

// Walks on from home bucket `hb` of a segment (a bucket full without the key)
// through the following buckets: the lane's slot found (bucket pointer in *at, lane
// returned), or -1 at the first empty slot or after every bucket.
__device__ __forceinline__ int walk_find(const Bucket* segb, uint32_t nb, uint32_t hb, int64_t key,
                                         BucketRegs* at) {
    const Bucket* b = segb + hb;
    for (uint32_t round = 1; round < nb; ++round) {
        b = b + 1 == segb + nb ? segb : b + 1;
        const BucketRegs v = load_bucket(b);
        bool end;
        const int l = bucket_find(v, key, &end);
        if (l >= 0) {
            *at = v;
            return l;
        }
        if (end) break;
    }
    return -1;
}

}  // namespace px
