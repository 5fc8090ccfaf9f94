/*
 * px.h - C ABI of the px library: GPU hash exchange, hash join and hash
 * aggregation over Arrow-layout columnar batches, for one NVIDIA GB300 (sm_103a).
 *
 * The operators restate those of the paper's GPU-aware Presto worker
 * ("Accelerating Presto with GPUs"): FilterProject's filter (Sec. 3.2),
 * PartitionedOutput's hash partitioning into per-destination queues that are
 * shipped as packed contiguous buffers with their sizes as metadata (Sec. 3.1,
 * Sec. 3.3.2), the join build and probe pipelines (Sec. 3.1, join-heavy Q5/Q9 of
 * Sec. 3.4), and HashAggregation in Single / Partial / Final modes (Sec. 3.2).
 * Data stay in device memory across operators (Sec. 2, hypotheses 2 and 3), and
 * each call is bound to a caller stream the way a CudfVector carries its stream
 * (Sec. 3.2).
 *
 * Conventions shared by every call
 *  - Columns are little-endian fixed-width signed integers (PX_I8, PX_I32,
 *    PX_I64) without validity buffers: nulls are not supported (TPC-H has none,
 *    Sec. 2.2). Every column base must be 16-byte aligned.
 *  - All pointers named d_* and every px_col.data are DEVICE pointers; the
 *    descriptor structs themselves (px_col, px_batch, px_agg arrays) are HOST
 *    memory and are only read during the call.
 *  - The library never allocates device memory and never synchronises, except
 *    px_stream_status. Callers pass every buffer, including a workspace `d_ws`
 *    sized by the matching px_*_ws_bytes query. A workspace may be reused by
 *    calls issued in order on one stream; calls that may overlap need distinct
 *    workspaces.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *    default stream). Inputs must stay valid until the stream work completes.
 *  - Host-checkable errors (null pointers, unknown types, misaligned columns,
 *    too-small workspaces, unsupported sizes) return PX_ERR_INVALID or
 *    PX_ERR_UNSUPPORTED immediately and launch nothing; px_last_error() gives a
 *    message. Data-dependent errors (an output over capacity, a duplicate build
 *    key, a full table, a bounded device wait that ran out) are recorded in the
 *    workspace's sticky status word (the first error wins) and are returned by
 *    px_stream_status. No call traps or faults the device on bad data: output
 *    rows past a capacity are not written, but the device row counts still
 *    report the size that would have been needed, so the caller can resize and
 *    retry. This is the paper's fail-rather-than-spill contract (Sec. 3.7).
 *  - Row counts: a batch has a host row count `nrows`; when `d_nrows` is set it
 *    is a device-resident actual count (<= nrows) and `nrows` is only the
 *    capacity. This lets operators chain on one stream without a host round
 *    trip for variable-size results. Row counts are below 2^31.
 *  - A selection (d_sel, d_nsel) lists, in ascending order, the input rows an
 *    operator reads; its entries are "positions" 0..*d_nsel-1. Without a
 *    selection the positions are the rows 0..n-1.
 *  - Segments (d_seg, nsegs) split the positions into nsegs consecutive ranges
 *    [d_seg[q], d_seg[q+1]) with d_seg[0] = 0 and d_seg[nsegs] = the position
 *    count; px_partition's d_offsets are exactly such segments. nsegs = 0 means
 *    one segment covering everything.
 */
#ifndef PX_H
#define PX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
typedef int32_t px_status;
#define PX_OK 0
#define PX_ERR_INVALID 1        /* bad argument (host check)                          */
#define PX_ERR_CAPACITY 2       /* an output exceeded its capacity (device status)    */
#define PX_ERR_DUPLICATE_KEY 3  /* duplicate key in a unique join build               */
#define PX_ERR_TABLE_FULL 4     /* a hash table ran out of slots                      */
#define PX_ERR_TIMEOUT 5        /* a bounded device-side wait gave up                 */
#define PX_ERR_CUDA 6           /* a CUDA runtime call failed                         */
#define PX_ERR_UNSUPPORTED 7    /* valid but unsupported (e.g. too many partitions)   */

/* ---- column types: the value is the element width in bytes -------------- */
#define PX_I8 1
#define PX_I32 4
#define PX_I64 8

/* A column: element type and device data pointer (16-byte aligned). */
typedef struct {
    int32_t type;      /* PX_I8, PX_I32 or PX_I64 */
    int32_t reserved;  /* must be 0 */
    void* data;        /* device pointer */
} px_col;

/* A columnar batch (Arrow fixed-width columns of equal length). */
typedef struct {
    int32_t ncols;
    int32_t reserved;        /* must be 0 */
    const px_col* cols;      /* host array of ncols descriptors */
    int64_t nrows;           /* row count, or capacity when d_nrows is set */
    const int64_t* d_nrows;  /* optional device row count (<= nrows); NULL: nrows */
} px_batch;

/* Aggregates (64-bit two's complement, wrapping mod 2^64; inputs sign-extended). */
#define PX_COUNT 0    /* COUNT(*)              */
#define PX_SUM 1      /* SUM(col[a])           */
#define PX_SUM_MUL 2  /* SUM(col[a] * col[b])  */
typedef struct {
    int32_t op;  /* PX_COUNT, PX_SUM or PX_SUM_MUL                 */
    int32_t a;   /* input column index (unused for PX_COUNT)       */
    int32_t b;   /* second input column index (PX_SUM_MUL only)    */
} px_agg;

/* Limits. */
#define PX_MAX_COLS 16
#define PX_MAX_PARTS 1024
#define PX_MAX_KEYS 2
#define PX_MAX_AGGS 8
#define PX_MAX_SEGS 4096

/* ---- workspace and status ----------------------------------------------- */

/* Zero the workspace's status word (and the rest of its header). Call once after
 * allocating a workspace, and again to clear a reported error. */
px_status px_ws_init(void* d_ws, size_t ws_bytes, void* stream);

/* Synchronise `stream`, then return the workspace's sticky status word: PX_OK or
 * the first data-dependent error recorded by a call that used d_ws. Returns
 * PX_ERR_CUDA if the stream reported a CUDA error. */
px_status px_stream_status(void* stream, const void* d_ws);

/* Thread-local message describing the last error returned by a call on this
 * thread ("" if none). Valid until the next call on the same thread. */
const char* px_last_error(void);

/* Instrumentation (the paper has no counterpart): number of CUDA kernels this
 * library has launched in the process so far, across all threads. Memsets and
 * copies are not counted. */
uint64_t px_kernel_launches(void);

/* Self-test of the bounded device waits (the paper has no counterpart): one
 * device thread polls the device int32 *d_flag (acquire loads, short sleeps)
 * until it is nonzero, giving up after spin_limit polls (1..2^24); the device
 * int32 *d_status receives PX_OK if the flag was seen set, PX_ERR_TIMEOUT if the
 * wait ran out. Every device-side wait in this library has this shape - bounded,
 * then a status word and a normal return - so a wait that nothing satisfies
 * never hangs or faults the device, and the context stays usable. */
px_status px_selftest_wait(const int32_t* d_flag, uint32_t spin_limit, int32_t* d_status, void* stream);

/* ---- filter (FilterProject's predicate, Sec. 3.2) ----------------------- */

size_t px_filter_ws_bytes(int64_t nrows);

/* Selection of the rows i < n with lo <= col[i] < hi (half-open), where n is
 * *d_nrows if given, else nrows. Writes the passing row indices in ascending order
 * to d_sel (capacity nrows) and their count to *d_nsel. col: PX_I8/I32/I64. */
px_status px_filter(const px_col* col, int64_t nrows, const int64_t* d_nrows,
                    int64_t lo, int64_t hi, int32_t* d_sel, int64_t* d_nsel,
                    void* d_ws, size_t ws_bytes, void* stream);

/* Allocation-free px_filter. The paper has no counterpart: this entry point is for
 * callers that cannot allocate device memory and so cannot pass a workspace - for
 * instance code embedded in a host engine whose memory manager owns every device
 * byte, or a serving loop that reserves all memory at start-up and must not call
 * cudaMalloc (which may synchronise the device) while serving. Same arguments and
 * results as px_filter, except that its scratch lives in one static device array
 * of 262,400 bytes inside this library (held by every GPU that loads it until the
 * process exits), so nrows may not exceed PX_FILTER_NOALLOC_MAX_ROWS
 * (PX_ERR_UNSUPPORTED otherwise; use px_filter). It allocates nothing. d_status
 * (nullable, device int32) receives the call's device status, which is always
 * PX_OK (the filter records no data-dependent error); it is kept so callers handle
 * every entry point alike. The first call on each device looks up the array's
 * device address on that device (cudaGetSymbolAddress) and caches it; make that
 * first call before any stream capture. Every call on a device shares the one
 * array (it keeps the last call's contents; each call writes every count it reads
 * before reading it), so calls whose GPU work may overlap (other streams, other
 * threads) race and must be serialised by the caller. */
#define PX_FILTER_NOALLOC_MAX_ROWS 134217728LL /* 65536 tiles of 2048 rows */
px_status px_filter_noalloc(const px_col* col, int64_t nrows, const int64_t* d_nrows,
                            int64_t lo, int64_t hi, int32_t* d_sel, int64_t* d_nsel,
                            int32_t* d_status, void* stream);

/* ---- hash partition: the on-device exchange (Sec. 3.1, Sec. 3.3.2) ------ */

size_t px_partition_ws_bytes(int64_t nrows, int32_t nparts);

/* Repartition the rows named by the positions of `in` (all rows, or the
 * selection d_sel/d_nsel) by the hash of the PX_I64 column key_col into nparts
 * (1..PX_MAX_PARTS) partitions. Row r goes to partition
 *     p(r) = floor(hi32(fmix64(key[r] XOR seed)) * nparts / 2^32)
 * (fmix64 = MurmurHash3's 64-bit finalizer; hi32 = its upper 32 bits). Every
 * column of `in` is written to the same-index column of `out` (same types,
 * capacity out->nrows >= the position count): partition 0's rows first, then
 * partition 1's, ..., each partition's rows in their input order (stable). This
 * is the packed per-destination buffer of the exchange; d_offsets[q] (nparts+1
 * int64) is the start of partition q and d_offsets[nparts] the row count - the
 * size metadata sent ahead of the data. out->d_nrows is ignored. */
px_status px_partition(const px_batch* in, int32_t key_col,
                       const int32_t* d_sel, const int64_t* d_nsel,
                       int32_t nparts, uint64_t seed, const px_batch* out,
                       int64_t* d_offsets, void* d_ws, size_t ws_bytes, void* stream);

/* Launch shape of px_partition: rows per thread in a tile of 256 threads (2, 4 or
 * 8, capped at the widest whose tile of every column fits the 48 KB staging
 * area; 0 = that widest) and the most resident scatter blocks per SM (0 = as many
 * as fit). Every shape gives the same result; they differ only in speed (an
 * autotuner picks one per GPU and workload). */
typedef struct {
    int32_t items;
    int32_t blocks_per_sm;
} px_partition_config;

/* px_partition with an explicit launch shape (cfg NULL = the defaults). */
px_status px_partition_tuned(const px_batch* in, int32_t key_col,
                             const int32_t* d_sel, const int64_t* d_nsel,
                             int32_t nparts, uint64_t seed, const px_batch* out,
                             int64_t* d_offsets, const px_partition_config* cfg,
                             void* d_ws, size_t ws_bytes, void* stream);

/* ---- hash join build (join build pipeline, Sec. 3.1) -------------------- */

/* Bytes of a join table for up to nbuild build rows in nsegs segments. */
size_t px_join_table_bytes(int64_t nbuild, int32_t nsegs);
size_t px_join_build_ws_bytes(int64_t nbuild);

/* Build an open-addressing hash table over the PX_I64 key column pk_col of
 * `build` (rows 0..n-1, n = *build->d_nrows or build->nrows), mapping each key to
 * its build row index. With nsegs > 0 the rows are split by d_seg (e.g. the
 * offsets px_partition wrote) into independent per-segment tables that a
 * segmented probe uses per partition. unique = 1 declares keys unique: a repeated
 * key records PX_ERR_DUPLICATE_KEY. unique = 0 keeps every row (multi-map). The
 * key value INT64_MIN is reserved as the empty-slot marker: a build key equal to
 * it records PX_ERR_UNSUPPORTED (probe keys equal to it never match). d_table
 * (table_bytes >= px_join_table_bytes) is caller memory with a private layout; it
 * stays valid for probes until rebuilt or freed. pay_col >= 0 (a PX_I8 or PX_I32
 * column of `build`, not pk_col) is copied into the table beside each key: a probe
 * whose build_payload is that one column (same address and type) reads the copy,
 * i.e. the column's values at build time, in the same memory access as the key,
 * instead of gathering them; pay_col = -1 copies nothing. */
px_status px_join_build(const px_batch* build, int32_t pk_col,
                        const int64_t* d_seg, int32_t nsegs, int32_t unique, int32_t pay_col,
                        void* d_table, size_t table_bytes,
                        void* d_ws, size_t ws_bytes, void* stream);

/* ---- hash join probe (join probe pipeline, Sec. 3.1; Q9 Sec. 3.4) ------- */

size_t px_join_probe_ws_bytes(int64_t nprobe);

/* Inner equi-join: for each position of `probe` (all rows or d_sel/d_nsel), in
 * position order, find the build rows whose key equals probe key column fk_col
 * (PX_I64) and emit one output row per match: the probe columns listed in
 * carry[0..ncarry) followed by all columns of build_payload (a batch indexed by
 * build row, e.g. the build batch itself; may be NULL) gathered at the matched
 * build row. out->ncols = ncarry + build_payload->ncols with matching types and
 * capacity out->nrows. Optional d_probe_row / d_build_row (int32, capacity
 * out->nrows) receive the matched probe and build row indices. *d_nout receives
 * the number of matches; over capacity, PX_ERR_CAPACITY is recorded and only the
 * first out->nrows are written. Output is in probe-position order; with a unique
 * build each probe row has at most one match. With nsegs > 0 (must equal the
 * table's) positions [d_seg[q], d_seg[q+1]) probe only segment q of the table, and
 * d_out_seg (nullable, nsegs+1 int64) receives the output segment offsets. */
px_status px_join_probe(const void* d_table, const px_batch* probe, int32_t fk_col,
                        const int32_t* d_sel, const int64_t* d_nsel,
                        const int64_t* d_seg, int32_t nsegs,
                        const int32_t* carry, int32_t ncarry,
                        const px_batch* build_payload, const px_batch* out,
                        int32_t* d_probe_row, int32_t* d_build_row,
                        int64_t* d_nout, int64_t* d_out_seg,
                        void* d_ws, size_t ws_bytes, void* stream);

/* ---- gather (late materialization, Sec. 2.3) ---------------------------- */
/* out->cols[c][i] = in->cols[c][d_idx[i]] for the positions i < n (n = *d_n when
 * given, else out->nrows): fetch payload columns by row id after the exchange and
 * join moved only (key, row id). Types must match per column; an index outside
 * [0, in->nrows) records PX_ERR_INVALID and that output row is left unwritten. */
px_status px_gather(const px_batch* in, const int32_t* d_idx, const int64_t* d_n, const px_batch* out,
                    void* d_ws, size_t ws_bytes, void* stream);

/* ---- hash aggregation (HashAggregation, Sec. 3.2) ----------------------- */

size_t px_groupby_ws_bytes(int64_t nrows, int64_t max_groups);

/* Optional column statistics for px_groupby_agg: key column k is expected (not
 * required) to lie in [lo[k], hi[k]], as a query engine knows from its catalog or
 * a dictionary. When the product of the ranges is small, each block aggregates
 * into dense shared-memory arrays indexed by the key instead of a hash table.
 * Rows outside the ranges are still aggregated exactly, through the hash path, so
 * a wrong range costs speed, never correctness. */
typedef struct {
    int64_t lo[PX_MAX_KEYS];
    int64_t hi[PX_MAX_KEYS];
} px_key_range;

/* GROUP BY the key columns key_cols[0..nkeys) (1..PX_MAX_KEYS columns of `in`)
 * over its positions (all rows or d_sel/d_nsel), computing aggs[0..naggs). With
 * nsegs > 0 groups are formed per segment (Partial aggregation per partition) and
 * d_out_seg (int32, capacity max_groups) receives each group's segment. Output
 * `out`: nkeys key columns (same types as the input keys) then naggs PX_I64
 * columns, capacity out->nrows >= max_groups; groups come in an unspecified
 * order. *d_ngroups receives the number of groups; more than max_groups records
 * PX_ERR_CAPACITY. The sum of the key widths plus ceil(log2(nsegs)) bits must not
 * exceed 64 bits (PX_ERR_UNSUPPORTED otherwise). `range` (nullable) is the key
 * statistic described above. A Final merge of Partial results is another
 * px_groupby_agg over them with PX_SUM of each partial aggregate. */
px_status px_groupby_agg(const px_batch* in, const int32_t* key_cols, int32_t nkeys,
                         const px_agg* aggs, int32_t naggs,
                         const int32_t* d_sel, const int64_t* d_nsel,
                         const int64_t* d_seg, int32_t nsegs, const px_key_range* range,
                         int64_t max_groups, const px_batch* out, int32_t* d_out_seg,
                         int64_t* d_ngroups, void* d_ws, size_t ws_bytes, void* stream);

/* Fused join probe + aggregation (the probe pipeline feeding HashAggregation in
 * Single, or per segment Partial, mode; Sec. 3.1, Sec. 3.2): the same groups as
 * px_join_probe (unique table, carrying the probe columns the aggregates read and
 * the build column `group` as payload) followed by px_groupby_agg grouping by that
 * payload column with key statistic [group_lo, group_hi], but without writing
 * the join output. aggs index the columns of `probe`; out = the group key column
 * (group->type) then naggs PX_I64 columns, capacity max_groups; with nsegs > 0
 * (must equal the table's) groups are per segment and d_out_seg receives each
 * group's segment. The statistic must be small enough for dense aggregation
 * (PX_ERR_UNSUPPORTED otherwise); group keys outside it are still aggregated
 * exactly. A multi-map table records PX_ERR_UNSUPPORTED. Groups come in an
 * unspecified order. */
size_t px_join_probe_agg_ws_bytes(int64_t nprobe, int64_t max_groups);
px_status px_join_probe_agg(const void* d_table, const px_batch* probe, int32_t fk_col,
                            const int32_t* d_sel, const int64_t* d_nsel,
                            const int64_t* d_seg, int32_t nsegs,
                            const px_col* group, int64_t nbuild, int64_t group_lo, int64_t group_hi,
                            const px_agg* aggs, int32_t naggs,
                            int64_t max_groups, const px_batch* out, int32_t* d_out_seg,
                            int64_t* d_ngroups, void* d_ws, size_t ws_bytes, void* stream);

/* Streaming aggregation (HashAggregation's Partial mode flushing its groups when
 * they pass a size threshold, and a Final that keeps merging them, Sec. 3.2): the
 * same call as px_groupby_agg plus flags.
 *   PX_AGG_STREAM      the call starts a stream of calls that share d_ws and the
 *                      outputs: the aggregation mode then depends on the key
 *                      statistic and max_groups only, not on the row count, so
 *                      every call of the stream keeps its groups in one place.
 *   PX_AGG_ACCUMULATE  continue the stream: add this call's rows into the groups
 *                      the earlier calls left in d_ws and the outputs (same keys,
 *                      aggregates, statistic, segments count, max_groups and
 *                      workspace) instead of starting empty. *d_ngroups and the
 *                      first *d_ngroups output rows then cover every call so far.
 * flags = 0 is px_groupby_agg. Emitting a Partial stream's groups into a Final
 * stream is another px_groupby_agg_stream over the Partial outputs with
 * d_nrows = its group count; the Partial stream then restarts without
 * PX_AGG_ACCUMULATE. */
#define PX_AGG_ACCUMULATE 1
#define PX_AGG_STREAM 2
px_status px_groupby_agg_stream(const px_batch* in, const int32_t* key_cols, int32_t nkeys,
                                const px_agg* aggs, int32_t naggs,
                                const int32_t* d_sel, const int64_t* d_nsel,
                                const int64_t* d_seg, int32_t nsegs, const px_key_range* range,
                                int64_t max_groups, const px_batch* out, int32_t* d_out_seg,
                                int64_t* d_ngroups, int32_t flags, void* d_ws, size_t ws_bytes,
                                void* stream);

/* ---- batched fused fragments: filter -> probe -> aggregate ------------- */
/* The paper runs many small plan fragments whose vectors are too small to fill a
 * GPU (Sec. 3.3.2; batch-size sensitivity, Sec. 3.4). This entry point runs a
 * batch of independent Q5/Q9-shaped fragments (FilterProject -> join probe ->
 * HashAggregation in Single mode) in ONE persistent kernel that pulls
 * (fragment, row chunk) work items from a device counter, plus one emit kernel.
 *
 * Fragment f: over its probe rows i < nrows keep those with
 * filter.lo <= filter[i] < filter.hi (all rows when filter.data is NULL), look
 * key[i] up in d_table (a unique, unsegmented table from px_join_build), and for
 * every match with build row r GROUP BY group[r] (a build-side column indexed by
 * build row), computing aggs over the probe columns cols[] (px_agg.a / .b index
 * cols). group_lo..group_hi is REQUIRED and is a guarantee (unlike px_key_range):
 * a matched row whose group key lies outside records PX_ERR_UNSUPPORTED and is
 * skipped. Results: the groups in ascending key order, keys in d_out_keys (type
 * group.type) and aggregates in d_out_aggs[a] (PX_I64), capacity max_groups;
 * *d_ngroups receives the group count (over capacity: PX_ERR_CAPACITY, first
 * max_groups written). A fragment's result does not depend on the other fragments
 * of the batch or on the configuration. */
#define PX_FRAG_MAX_COLS 4
#define PX_FRAG_MAX_AGGS 4
#define PX_FRAG_MAX_GROUPS (1LL << 22) /* group_hi - group_lo + 1 at most */
typedef struct {
    int64_t nrows;                            /* probe rows (< 2^31) */
    px_col key;                               /* PX_I64 join key */
    px_col filter;                            /* PX_I8/I32/I64; data NULL: no filter */
    int64_t lo, hi;                           /* keep lo <= filter < hi */
    int32_t ncols;                            /* 0..PX_FRAG_MAX_COLS */
    int32_t naggs;                            /* 0..PX_FRAG_MAX_AGGS */
    px_col cols[PX_FRAG_MAX_COLS];            /* probe columns the aggregates read */
    px_agg aggs[PX_FRAG_MAX_AGGS];
    const void* d_table;                      /* unique, unsegmented join table */
    int64_t nbuild;                           /* build rows: the length of group */
    px_col group;                             /* build column: the group key */
    int64_t group_lo, group_hi;               /* every group key lies in [group_lo, group_hi] */
    int64_t max_groups;                       /* output capacity */
    void* d_out_keys;                         /* group.type, capacity max_groups */
    int64_t* d_out_aggs[PX_FRAG_MAX_AGGS];    /* PX_I64, capacity max_groups each */
    int64_t* d_ngroups;                       /* device int64 */
} px_fragment;

/* Launch configuration of px_fragments_run (NULL: library defaults). threads per
 * block (256 or 512), items per thread (2 or 4), rows per work item (a multiple
 * of threads * items, or 0: chosen from the batch's total rows so that the
 * persistent grid gets about four items per block, within [one tile, 65536];
 * fragments whose dense accumulators live in shared memory take at least 4 group
 * slots' worth of rows per item), and resident blocks per SM of the persistent
 * grid (1..8; capped by what fits). A project autotuner picks these per GPU;
 * every configuration gives the same results. */
typedef struct {
    int32_t threads;
    int32_t items;
    int64_t chunk_rows;
    int32_t blocks_per_sm;
} px_fragments_config;

/* Host staging bytes for the plan of nfrags fragments (see px_fragments_run). */
size_t px_fragments_plan_bytes(int32_t nfrags);
size_t px_fragments_ws_bytes(const px_fragment* frags, int32_t nfrags);

/* Run nfrags fragments as one batch. h_plan (px_fragments_plan_bytes bytes, HOST
 * memory, pinned for an asynchronous upload) receives the device plan, which is
 * copied into d_ws on `stream`; it must stay unchanged until the stream work has
 * completed. */
px_status px_fragments_run(const px_fragment* frags, int32_t nfrags, const px_fragments_config* cfg,
                           void* h_plan, size_t plan_bytes, void* d_ws, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PX_H */
