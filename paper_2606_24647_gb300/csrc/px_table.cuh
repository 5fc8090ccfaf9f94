// Join hash table layout shared by the join (px_join.cu) and the fused fragment
// pipelines (px_fragments.cu). The table is caller memory:
//   [0, 64)            header: magic, nsegs, unique flag, build rows
//   [64, 64 + A)       copy of the build segment offsets (nsegs + 1 int64)
//   [64 + A + p, ...)  buckets of 64 bytes: 4 int64 keys, their 4 int32 build
//                      rows, 16 bytes of padding; p < 64 pads the first bucket
//                      to a 64-byte address (the caller's table is only 16-byte
//                      aligned), so 32-byte vector loads of a bucket's keys are
//                      aligned
// Segment q of n_q rows owns buckets [b_q, b_{q+1}) with b_q = floor(seg[q] / 2) + q
// (at least 2 n_q + 2 slots: load factor < 1/2). Slots are numbered
// 4 * bucket + lane; linear probing over slots starts at the first slot of the
// key's home bucket. Empty slots hold the key INT64_MIN.
#pragma once

#include "px_common.cuh"

namespace px {

constexpr int64_t kEmpty = INT64_MIN;
constexpr int64_t kMagic = 0x707874626c763032ll;  // "pxtblv02"

struct TableHeader {
    int64_t magic;
    int32_t nsegs;   // >= 1
    int32_t unique;
    int64_t nbuild;  // build rows inserted
    int64_t reserved[5];
};

struct Bucket {
    int64_t key[4];
    int32_t row[4];
    int32_t pad[4];
};
static_assert(sizeof(Bucket) == 64, "bucket is one half of a 128-byte line");

inline size_t seg_area_bytes(int32_t S) { return align_up(static_cast<size_t>(S + 1) * 8, 64); }
__host__ __device__ inline int64_t table_buckets(int64_t n, int32_t S) { return n / 2 + S; }

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
    t.bk = reinterpret_cast<Bucket*>((bk + 63) & ~static_cast<uintptr_t>(63));
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
    g.b0 = s0 / 2 + q;
    g.nb = static_cast<uint32_t>(s1 / 2 - s0 / 2 + 1);
    return g;
}

__device__ __forceinline__ uint32_t home_bucket(uint64_t key, uint32_t nb) { return slot_of(fmix64(key), nb); }

// Looks `key` up in the 4 keys k01, k23 of one bucket: the lane of the match, or
// -1 with *end set when an empty slot ends the probe sequence in this bucket.
// Occupied slots form a prefix of every probe sequence (inserts take the first
// empty slot), so a present key precedes the first empty slot. Branch-free.
__device__ __forceinline__ int bucket_find(longlong2 k01, longlong2 k23, int64_t key, bool* end) {
    const int l = k01.x == key ? 0 : (k01.y == key ? 1 : (k23.x == key ? 2 : (k23.y == key ? 3 : -1)));
    *end = l < 0 && (k01.x == kEmpty || k01.y == kEmpty || k23.x == kEmpty || k23.y == kEmpty);
    return l;
}

}  // namespace px
