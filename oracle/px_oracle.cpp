// px oracle: TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded CPU statement of what the GPU operators compute:
// filter, hash partition (the on-device exchange), equi-join and hash aggregation
// over Arrow fixed-width int8/int32/int64 columns without nulls (Sec. 2.2: TPC-H has
// no nulls, so none are modelled). Only the test suite, the smoke check and the
// bench's CPU-baseline / reference arm may load this library. It shares no code,
// header or constant table with the CUDA library; the two meet only on the seeded
// inputs drawn by pxdata.
//
// Operator statements followed (the paper describes the operators as Velox/cuDF
// operators and names no algorithm, so each function below is the SQL definition
// written out directly):
//   filter     - FilterProject evaluates the predicate and keeps passing rows
//                (Sec. 3.2). Predicate: lo <= col < hi (half-open reading).
//   partition  - PartitionedOutput splits each batch by key hash into one queue
//                per destination, each sent as one packed contiguous buffer with
//                its size as metadata (Sec. 3.1, Sec. 3.3.2). Reading: stable
//                order inside a partition, partition = multiply-shift range
//                reduction of the upper 32 bits of fmix64(key ^ seed).
//   join       - inner equi-join of probe rows against build rows (Sec. 3, join
//                pipelines; Q9/Q5 are the join-heavy queries of Sec. 3.4).
//                Reading: output in probe-position order, matches of one probe
//                row in ascending build-row order.
//   group-by   - HashAggregation in Single / Partial / Final modes (Sec. 3.2):
//                COUNT, SUM(a), SUM(a*b) in 64-bit two's complement (wrapping),
//                groups reported in ascending (segment, key...) order.
// Every one of these is pinned by the non-GPU tests against brute force,
// closed forms and invariants.
//
// Algorithms are chosen to differ from the GPU's: stable_sort for partition,
// sorted build keys + binary search for the join, std::map for the group-by.

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

namespace {

// Read element i of a little-endian fixed-width signed integer column.
int64_t load_int(const void* col, int32_t width, int64_t i) {
    switch (width) {
        case 1: return static_cast<int64_t>(static_cast<const int8_t*>(col)[i]);
        case 4: return static_cast<int64_t>(static_cast<const int32_t*>(col)[i]);
        case 8: return static_cast<const int64_t*>(col)[i];
        default: return 0;
    }
}

// Copy element `src_i` of `src` into element `dst_i` of `dst` (same width).
void copy_elem(void* dst, int64_t dst_i, const void* src, int64_t src_i, int32_t width) {
    std::memcpy(static_cast<char*>(dst) + dst_i * width,
                static_cast<const char*>(src) + src_i * width, static_cast<size_t>(width));
}

// Row index of probe/input position j: sel[j] when a selection vector is given.
int64_t row_at(const int32_t* sel, int64_t j) { return sel ? static_cast<int64_t>(sel[j]) : j; }

}  // namespace

extern "C" {

// MurmurHash3's 64-bit finalizer (A. Appleby, public domain): three xor-shifts by
// 33 bits interleaved with two multiplications by odd constants. A bijection on
// 64-bit words.
uint64_t orc_fmix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}

// Destination partition of a key: the upper 32 bits of fmix64(key ^ seed) mapped to
// [0, nparts) by Lemire's multiply-shift range reduction.
int32_t orc_part_of(int64_t key, uint64_t seed, int32_t nparts) {
    const uint64_t h = orc_fmix64(static_cast<uint64_t>(key) ^ seed);
    return static_cast<int32_t>(((h >> 32) * static_cast<uint64_t>(nparts)) >> 32);
}

// Filter: sel = ascending list of rows i with lo <= col[i] < hi. Returns its length.
int64_t orc_filter(const void* col, int32_t width, int64_t n, int64_t lo, int64_t hi,
                   int32_t* sel) {
    int64_t count = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t v = load_int(col, width, i);
        if (lo <= v && v < hi) sel[count++] = static_cast<int32_t>(i);
    }
    return count;
}

// Hash partition. Input positions j = 0..m-1 (m = nsel if sel else nrows) name rows
// row(j); each row goes to partition part_of(key[row]). Output: the rows stably
// sorted by partition (input order kept inside a partition), every column
// gathered in that order, and offsets[q] = number of rows in partitions < q
// (offsets[nparts] = m). Returns 0.
int32_t orc_partition(int32_t ncols, const int32_t* widths, const void* const* cols,
                      int64_t nrows, int32_t key_col, const int32_t* sel, int64_t nsel,
                      int32_t nparts, uint64_t seed, void* const* out_cols, int64_t* offsets) {
    const int64_t m = sel ? nsel : nrows;
    std::vector<int32_t> part(static_cast<size_t>(m));
    std::vector<int64_t> order(static_cast<size_t>(m));
    for (int64_t j = 0; j < m; ++j) {
        const int64_t key = load_int(cols[key_col], widths[key_col], row_at(sel, j));
        part[j] = orc_part_of(key, seed, nparts);
        order[j] = j;
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t a, int64_t b) { return part[a] < part[b]; });
    for (int32_t c = 0; c < ncols; ++c)
        for (int64_t o = 0; o < m; ++o)
            copy_elem(out_cols[c], o, cols[c], row_at(sel, order[o]), widths[c]);
    for (int32_t q = 0; q <= nparts; ++q) offsets[q] = 0;
    for (int64_t j = 0; j < m; ++j) offsets[part[j] + 1] += 1;
    for (int32_t q = 0; q < nparts; ++q) offsets[q + 1] += offsets[q];
    return 0;
}

// Inner equi-join fk = pk. Probe positions j = 0..m-1 (m = nsel if sel else nprobe)
// name probe rows row(j). With nsegs > 0 the join is done per segment: positions
// [probe_seg[q], probe_seg[q+1]) only meet build rows [build_seg[q], build_seg[q+1]).
// Output pairs (probe row, build row) in probe-position order, the matches of one
// probe row in ascending build-row order; the first `cap` are written. When
// out_seg is given, out_seg[q] = number of output pairs from segments < q.
// Returns the total number of pairs.
int64_t orc_join(const int64_t* pk, int64_t nbuild, const int64_t* build_seg,
                 const int64_t* fk, int64_t nprobe, const int32_t* sel, int64_t nsel,
                 const int64_t* probe_seg, int32_t nsegs, int64_t cap,
                 int32_t* probe_row, int32_t* build_row, int64_t* out_seg) {
    const int64_t m = sel ? nsel : nprobe;
    const int32_t S = nsegs > 0 ? nsegs : 1;
    int64_t nout = 0;
    for (int32_t q = 0; q < S; ++q) {
        const int64_t b0 = nsegs > 0 ? build_seg[q] : 0;
        const int64_t b1 = nsegs > 0 ? build_seg[q + 1] : nbuild;
        const int64_t p0 = nsegs > 0 ? probe_seg[q] : 0;
        const int64_t p1 = nsegs > 0 ? probe_seg[q + 1] : m;
        if (out_seg) out_seg[q] = nout;
        // Sorted (key, build row) pairs of this segment's build side.
        std::vector<std::pair<int64_t, int64_t>> sorted;
        sorted.reserve(static_cast<size_t>(b1 - b0));
        for (int64_t b = b0; b < b1; ++b) sorted.emplace_back(pk[b], b);
        std::sort(sorted.begin(), sorted.end());
        for (int64_t j = p0; j < p1; ++j) {
            const int64_t r = row_at(sel, j);
            const int64_t key = fk[r];
            auto lo = std::lower_bound(sorted.begin(), sorted.end(),
                                       std::make_pair(key, INT64_MIN));
            for (auto it = lo; it != sorted.end() && it->first == key; ++it) {
                if (nout < cap) {
                    probe_row[nout] = static_cast<int32_t>(r);
                    build_row[nout] = static_cast<int32_t>(it->second);
                }
                ++nout;
            }
        }
    }
    if (out_seg) out_seg[S] = nout;
    return nout;
}

// Hash aggregation. Positions j = 0..m-1 name rows row(j); with nsegs > 0 position j
// belongs to the segment q with seg[q] <= j < seg[q+1] and groups are formed per
// segment (Partial mode per partition); otherwise every row is in segment 0.
// Group key = (segment, key columns...), compared as signed integers,
// lexicographically. Aggregates: op 0 COUNT(*), op 1 SUM(a), op 2 SUM(a*b), all in
// 64-bit two's complement arithmetic (wrapping mod 2^64).
// Output: groups in ascending key order; the first max_groups are written:
// out_seg[g] (if non-null), out_keys[k * max_groups + g], out_aggs[a * max_groups + g].
// Returns the number of groups.
int64_t orc_groupby(int64_t nrows, const int32_t* sel, int64_t nsel,
                    const int64_t* seg, int32_t nsegs,
                    int32_t nkeys, const int32_t* key_widths, const void* const* key_cols,
                    int32_t naggs, const int32_t* ops,
                    const int32_t* a_widths, const void* const* a_cols,
                    const int32_t* b_widths, const void* const* b_cols,
                    int64_t max_groups, int32_t* out_seg, int64_t* out_keys,
                    int64_t* out_aggs) {
    const int64_t m = sel ? nsel : nrows;
    std::map<std::vector<int64_t>, std::vector<uint64_t>> groups;
    int32_t q = 0;
    for (int64_t j = 0; j < m; ++j) {
        if (nsegs > 0)
            while (q + 1 < nsegs && j >= seg[q + 1]) ++q;
        const int64_t r = row_at(sel, j);
        std::vector<int64_t> key;
        key.push_back(nsegs > 0 ? q : 0);
        for (int32_t k = 0; k < nkeys; ++k) key.push_back(load_int(key_cols[k], key_widths[k], r));
        std::vector<uint64_t>& acc = groups[key];
        if (acc.empty()) acc.assign(static_cast<size_t>(naggs), 0);
        for (int32_t a = 0; a < naggs; ++a) {
            if (ops[a] == 0) {
                acc[a] += 1;
            } else if (ops[a] == 1) {
                acc[a] += static_cast<uint64_t>(load_int(a_cols[a], a_widths[a], r));
            } else {
                const uint64_t x = static_cast<uint64_t>(load_int(a_cols[a], a_widths[a], r));
                const uint64_t y = static_cast<uint64_t>(load_int(b_cols[a], b_widths[a], r));
                acc[a] += x * y;
            }
        }
    }
    int64_t g = 0;
    for (const auto& kv : groups) {
        if (g < max_groups) {
            if (out_seg) out_seg[g] = static_cast<int32_t>(kv.first[0]);
            for (int32_t k = 0; k < nkeys; ++k) out_keys[k * max_groups + g] = kv.first[k + 1];
            for (int32_t a = 0; a < naggs; ++a)
                out_aggs[a * max_groups + g] = static_cast<int64_t>(kv.second[a]);
        }
        ++g;
    }
    return g;
}

}  // extern "C"
