/*
 * tqp.h -- C ABI of the B300 (sm_103a) key-sort-and-segment core of a tensor
 * query processor.
 *
 * The paper ("Share the Tensor Tea", VLDB 2022) represents every table column
 * as an (n x 1) tensor of numbers (Section 2.1) and compiles relational
 * operators -- filters, joins, aggregations -- into programs over those
 * column tensors (Section 2.2); its evaluation runs a filter-plus-aggregation
 * query (TPC-H Q6) and a join-plus-aggregation query (Q14) (Section 2.3).
 * This library implements those operators directly as CUDA kernels over
 * integer column vectors: filter by stream compaction, stable LSD radix sort,
 * sort-based equi-join (bound search + expand), sort-based group-by with
 * exact 64-bit aggregates, a fused star-join aggregate, a learned range
 * partitioner (a small monotone network trained on the GPU, after the
 * paper's Section 3.3 in-query neural network inference), and batched
 * launches of many small instances.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers named d_* and all column data are DEVICE pointers on the
 *    current CUDA device; arrays of descriptors (tqp_col, tqp_pred, ...) are
 *    HOST memory read during the call.  The library never takes ownership of
 *    a pointer, never allocates or frees device memory, and never
 *    synchronises the stream (except tqp_status_poll).  All work is enqueued
 *    on the given stream (0 = legacy default stream).
 *  - Workspace: every call that needs scratch takes (ws, ws_bytes).  Call it
 *    first with ws == NULL: it writes the bytes it needs to *ws_bytes, does
 *    nothing else and returns TQP_OK.  Then call again with a device buffer
 *    of at least that size, 256-byte aligned (a misaligned workspace is
 *    refused with TQP_ERR_INVALID before any work).  The size depends only on the
 *    host arguments (sizes, counts, dtypes), not on the data.
 *  - Row counts: n is the (maximum) row count known on the host.  Where an
 *    argument d_n is accepted, a non-NULL d_n points to a device int64 that
 *    holds the actual count (<= n), e.g. the result count of an earlier
 *    filter; the kernels read it on the device, so chains of calls need no
 *    host synchronisation and can be captured in a CUDA graph.
 *  - Result counts (d_out_n, d_out_groups) are written to device memory.  If
 *    a result does not fit in its capacity, the full required count is still
 *    written, only the first `cap` results are stored, and the device status
 *    word records TQP_ERR_CAPACITY.
 *  - Errors: argument errors are detected on the host before anything is
 *    launched and returned directly (TQP_ERR_INVALID / TQP_ERR_DTYPE /
 *    TQP_ERR_WORKSPACE / TQP_ERR_UNSUPPORTED).  A failed launch returns
 *    TQP_ERR_CUDA.  Errors found on the device (capacity, a bounded wait that
 *    ran out, a key wider than 64 packed bits) are recorded in a per-device
 *    status word (first error wins) that tqp_status_poll returns and clears.
 *  - Limits: n < 2^30 rows per call for sorts and group-bys, n < 2^31 for
 *    filters, gathers and joins (row ids are int32).
 *  - Signed semantics: keys and values are two's-complement signed integers;
 *    key order is ascending signed order.  Aggregates are exact 64-bit
 *    integers; SUM wraps modulo 2^64.
 */
#ifndef TQP_H_
#define TQP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* tqp_stream_t; /* same type as cudaStream_t */

typedef enum {
  TQP_OK = 0,
  TQP_ERR_INVALID = 1,     /* bad argument (NULL pointer, negative size, bad enum) */
  TQP_ERR_DTYPE = 2,       /* unsupported or mismatched column dtype */
  TQP_ERR_CAPACITY = 3,    /* (device) a result did not fit its capacity */
  TQP_ERR_CUDA = 4,        /* a CUDA launch or copy failed */
  TQP_ERR_TIMEOUT = 5,     /* (device) a bounded inter-block wait ran out */
  TQP_ERR_WORKSPACE = 6,   /* workspace smaller than the size query returned */
  TQP_ERR_UNSUPPORTED = 7, /* valid but unsupported (e.g. >64 packed key bits) */
  TQP_ERR_TOO_LARGE = 8    /* input larger than a fixed-size entry point accepts */
} tqp_status;

typedef enum { TQP_I8 = 1, TQP_I16 = 2, TQP_I32 = 3, TQP_I64 = 4 } tqp_dtype;

/* One column: an (n x 1) integer tensor (Section 2.1), device memory,
 * contiguous, not owned.  Its length is given by the call's n. */
typedef struct {
  const void* data;
  int32_t dtype; /* tqp_dtype */
  int32_t pad_;
} tqp_col;

typedef enum { TQP_LT = 0, TQP_LE = 1, TQP_GT = 2, TQP_GE = 3, TQP_EQ = 4, TQP_NE = 5 } tqp_cmp;

/* Predicate `cols[col] op lit`, the column's signed value against a signed
 * 64-bit literal.  Predicates of one call are AND-ed. */
typedef struct {
  int32_t col;
  int32_t op; /* tqp_cmp */
  int64_t lit;
} tqp_pred;

typedef enum { TQP_COUNT = 0, TQP_SUM = 1, TQP_MIN = 2, TQP_MAX = 3 } tqp_aggop;

/* Value expression: the product over its nterms (1..3) terms of
 * (mul * vals[col][row] + add), evaluated per row in 64-bit two's
 * complement.  E.g. price*(100-disc)*(100+tax) is three terms
 * {price,1,0} {disc,-1,100} {tax,1,100}. */
typedef struct {
  int32_t col;
  int32_t pad_;
  int64_t mul;
  int64_t add;
} tqp_term;

typedef struct {
  int32_t nterms;
  int32_t pad_;
  tqp_term term[3];
} tqp_expr;

/* One aggregate: op over expression exprs[expr] (ignored for COUNT). */
typedef struct {
  int32_t op; /* tqp_aggop */
  int32_t expr;
} tqp_agg;

#define TQP_MAX_PREDS 4
#define TQP_MAX_KEYS 4
#define TQP_MAX_VALS 8
#define TQP_MAX_EXPRS 8
#define TQP_MAX_AGGS 8

/* ------------------------------------------------------------------------
 * tqp_filter -- relational selection (Section 2.2; the Q6 filters of
 * Section 2.3) by single-pass stream compaction.
 * Writes the ascending int32 indices i (0 <= i < n, or < *d_n) of the rows
 * where every predicate holds to d_out_idx (capacity cap) and their count to
 * *d_out_n.  cols[k] are columns of n rows; npred in 0..TQP_MAX_PREDS (0 =
 * keep every row).
 * ---------------------------------------------------------------------- */
tqp_status tqp_filter(const tqp_col* cols, int ncols, const tqp_pred* preds, int npred,
                      int64_t n, const int64_t* d_n, int32_t* d_out_idx, int64_t cap,
                      int64_t* d_out_n, void* ws, size_t* ws_bytes, tqp_stream_t stream);

/* ------------------------------------------------------------------------
 * tqp_filter_noalloc -- the filter of tqp_filter for callers that cannot
 * provide a workspace.  The paper has no counterpart; this is a packaging
 * variant of the same kernel.
 *
 * Some callers cannot allocate device memory at all: a host program whose
 * own memory manager owns every device allocation and forbids others, or
 * code running where an allocation is not allowed or could stall (inside a
 * driver callback or a latency-critical loop).  They still own and pass the
 * inputs and the outputs (d_out_idx, d_out_n); only the scratch moves: the
 * kernel's look-back status words and tile counter live in a fixed array of
 * the library's device data (about 512 KiB, held by every GPU that loads the
 * library until the process exits).  Hence the size limit: n may not exceed
 * TQP_NOALLOC_MAX_ROWS, else TQP_ERR_TOO_LARGE is returned before any work.
 * The call allocates nothing and zeroes the scratch it uses on `stream`.
 * The first call on each device looks up the array's device address (done
 * once per device, with that device current); make that first call before
 * any stream capture.  Every call shares the one array: calls whose work
 * overlaps on the GPU (other streams, other threads) race and must be
 * serialised by the caller.  Arguments, results and errors otherwise as for
 * tqp_filter.
 * ---------------------------------------------------------------------- */
#define TQP_NOALLOC_MAX_ROWS (1LL << 28)
tqp_status tqp_filter_noalloc(const tqp_col* cols, int ncols, const tqp_pred* preds, int npred,
                              int64_t n, const int64_t* d_n, int32_t* d_out_idx, int64_t cap,
                              int64_t* d_out_n, tqp_stream_t stream);

/* ------------------------------------------------------------------------
 * tqp_gather -- column gather, d_out[j] = col[d_idx[j]] for j < n (or < *d_n),
 * in the column's dtype.  The caller guarantees every index is in range.
 * ---------------------------------------------------------------------- */
tqp_status tqp_gather(tqp_col col, const int32_t* d_idx, int64_t n, const int64_t* d_n,
                      void* d_out, tqp_stream_t stream);

/* ------------------------------------------------------------------------
 * tqp_like_prefix -- SQL `value LIKE 'prefix%'` over a string column held,
 * as Section 2.1 describes, in an (n x width) byte tensor: row i (width
 * bytes at d_str + i * width, row-major, device memory) holds the UTF-8
 * bytes of value i right-padded with zeros.  d_out[i] = 1 when the row's
 * first plen bytes equal prefix, else 0: an empty prefix matches every row;
 * a prefix longer than width matches none.  The result is an int8 column
 * that serves as a filter predicate column (d_out != 0) and, as a 0/1 value
 * term, turns an aggregate into SUM(CASE WHEN ... THEN expr ELSE 0 END).
 * prefix is host memory, copied at the call: plen <= 64 bytes, no zero byte.
 * width: 1..256.  Errors: TQP_ERR_INVALID for a bad size, a null pointer or
 * a zero byte in the prefix.  Rows are staged in shared memory with 16-byte
 * loads when d_str is 16-byte aligned.
 * ---------------------------------------------------------------------- */
tqp_status tqp_like_prefix(const uint8_t* d_str, int64_t n, int32_t width, const uint8_t* prefix, int32_t plen,
                           int8_t* d_out, tqp_stream_t stream);

/* ------------------------------------------------------------------------
 * tqp_string_codes -- dictionary codes of a string column (the same (n x
 * width) zero-padded byte tensor as tqp_like_prefix), for grouping or
 * ordering by a string: d_codes[i] = the rank of row i's value among the
 * column's distinct values in ascending byte order (the zero padding sorts a
 * value before every longer value it prefixes); d_rep_rows[c] = a row whose
 * value has code c, for c < *d_ncodes.  The rows are sorted as multi-word
 * keys (8-byte big-endian words, least significant first, each round a
 * stable radix sort), then numbered at each change of value.  Grouping by
 * d_codes with tqp_groupby_agg groups by the string, in string order.
 * n < 2^30, width 1..256.  Two-phase workspace sizing as for tqp_sort_pairs.
 * ---------------------------------------------------------------------- */
tqp_status tqp_string_codes(const uint8_t* d_str, int64_t n, int32_t width, int32_t* d_codes, int32_t* d_rep_rows,
                            int64_t* d_ncodes, void* ws, size_t* ws_bytes, tqp_stream_t stream);

/* ------------------------------------------------------------------------
 * Date columns (Section 2.1): a date is stored as its UNIX epoch time in
 * nanoseconds, an int64 column; a range predicate on dates is then two
 * predicates on that column.  The paper names dates (with strings) as the
 * columns whose ingestion needs a conversion; these calls do it on the GPU.
 * Calendar: proleptic Gregorian.  Int64 nanoseconds hold the whole days
 * -106751..106751 around 1970-01-01 (1677-09-22 to 2262-04-11).
 *
 * tqp_date_parse_iso: row i of an (n x width) zero-padded byte tensor (the
 *   string layout of tqp_like_prefix) holding "YYYY-MM-DD" (exactly ten
 *   bytes, then only zero bytes) -> d_ns[i] = the date's epoch ns.  A
 *   malformed row (bad digits or separators, a month or day that does not
 *   exist, a date outside the range above, other bytes after the date) gets
 *   INT64_MIN and the device status records TQP_ERR_INVALID.  width 10..256.
 * tqp_date_from_days: d_days[i] (days since 1970-01-01) -> d_ns[i]; a day
 *   outside the range gives INT64_MIN and records TQP_ERR_INVALID.
 * tqp_date_parts: d_ns[i] -> the day number floor(ns / 86400e9) (an instant
 *   before 1970 belongs to the earlier day), its year, month (1..12) and day
 *   of month (1..31); each output pointer may be NULL.
 * All: device pointers, n < 2^31, enqueued on `stream`; TQP_ERR_INVALID for
 * bad sizes or NULL inputs.
 * ---------------------------------------------------------------------- */
tqp_status tqp_date_parse_iso(const uint8_t* d_str, int64_t n, int32_t width, int64_t* d_ns, tqp_stream_t stream);
tqp_status tqp_date_from_days(const int32_t* d_days, int64_t n, int64_t* d_ns, tqp_stream_t stream);
tqp_status tqp_date_parts(const int64_t* d_ns, int64_t n, int32_t* d_days, int32_t* d_year, int32_t* d_month,
                          int32_t* d_mday, tqp_stream_t stream);

/* ------------------------------------------------------------------------
 * tqp_sort_pairs -- stable ascending LSD radix sort of (key, value) pairs
 * (the sort under the sort-based join and group-by of Section 2.2).
 * Keys (dtype TQP_I8..TQP_I64) are ordered by bits [begin_bit, end_bit) of
 * their order-preserving image (the sign bit flipped); (0, width) sorts by the
 * full signed value.  d_vals_in may be NULL: the payload is then the input
 * row index.  Ties keep input order.  Output buffers must not alias inputs.
 * ---------------------------------------------------------------------- */
tqp_status tqp_sort_pairs(int32_t key_dtype, const void* d_keys_in, const int32_t* d_vals_in,
                          void* d_keys_out, int32_t* d_vals_out, int64_t n, const int64_t* d_n,
                          int begin_bit, int end_bit, void* ws, size_t* ws_bytes,
                          tqp_stream_t stream);

/* ------------------------------------------------------------------------
 * tqp_join_eq -- inner equi-join (Section 2.2; the Q14 join of Section 2.3)
 * by sorting the build side and, per probe row, a bound search for the range
 * of equal keys, whose pairs are expanded in place.
 * Output: pairs (d_out_probe[k], d_out_build[k]) of row indices with
 * probe[i] == build[j], ordered by probe row, then build row; the count goes
 * to *d_out_n.  probe and build must share one dtype.
 * ---------------------------------------------------------------------- */
tqp_status tqp_join_eq(tqp_col probe, int64_t n_probe, const int64_t* d_n_probe, tqp_col build,
                       int64_t n_build, const int64_t* d_n_build, int32_t* d_out_probe,
                       int32_t* d_out_build, int64_t cap, int64_t* d_out_n, void* ws,
                       size_t* ws_bytes, tqp_stream_t stream);

/* ------------------------------------------------------------------------
 * tqp_groupby_agg -- sort-based group-by aggregation (Section 2.2; the
 * aggregates of Section 2.3 and the expression aggregate of Fig. 4).
 * Rows: d_sel[0..n) if d_sel is given, else 0..n-1 (n or *d_n).
 * Keys (1..TQP_MAX_KEYS columns) are packed into one order-preserving word
 * (each column trimmed to its [min, max] range), sorted, split into segments
 * of equal keys, and each segment reduced.  Output: G groups in ascending
 * lexicographic signed key order; d_out_keys[k] receives key column k (its
 * own dtype, capacity cap); d_out_aggs[g * naggs + a] the aggregates
 * (int64).  G goes to *d_out_groups.  The packed key must fit in 64 bits,
 * else the device status records TQP_ERR_UNSUPPORTED and G = 0.  A packed
 * key of at most 10 bits (decided on the device from the key range) is its
 * own group slot: the rows are folded into slot accumulators without the
 * sort, with the same results.  More than cap groups: the first cap are
 * written, G is the full count, and the status records TQP_ERR_CAPACITY.
 * ---------------------------------------------------------------------- */
tqp_status tqp_groupby_agg(const tqp_col* keys, int nkeys, const tqp_col* vals, int nvals,
                           const tqp_expr* exprs, int nexprs, const tqp_agg* aggs, int naggs,
                           const int32_t* d_sel, int64_t n, const int64_t* d_n,
                           void* const* d_out_keys, int64_t* d_out_aggs, int64_t cap,
                           int64_t* d_out_groups, void* ws, size_t* ws_bytes,
                           tqp_stream_t stream);

/* ------------------------------------------------------------------------
 * tqp_star_agg -- fused star join + filter + group-by aggregate (the Q14
 * shape of Section 2.3 generalised to up to two dimension tables):
 *   SELECT dim keys, aggs FROM fact JOIN dim_0 ON fact.fk_0 = dim_0.key
 *   [JOIN dim_1 ON fact.fk_1 = dim_1.key] WHERE fact_preds AND dim_preds
 *   GROUP BY (group key of dim_0, group key of dim_1).
 * Each dimension is filtered by its predicates, sorted on its key, and
 * grouped by its (optional) group column; each fact row then bound-searches
 * every dimension and folds its expression values into its group's
 * aggregates, without materialising join pairs.  Dimension keys must be
 * unique among the rows passing the dimension's predicates (a foreign-key
 * join); a duplicate is reported as TQP_ERR_UNSUPPORTED on the device.
 * Aggregate expressions read fact columns (val_src = 0) or a dimension's
 * value column (val_src = 1 + d).  Outputs as for tqp_groupby_agg with one
 * key column per dimension that has a group column.
 * ---------------------------------------------------------------------- */
typedef struct {
  tqp_col key;           /* dimension key (TQP_I32 or TQP_I64), n rows */
  int64_t n;
  tqp_col group;         /* group-by column, or data == NULL for none */
  const tqp_pred* preds; /* predicates over cols[] of this dimension */
  int npred;
  int ncols;
  const tqp_col* cols;   /* columns predicates and values refer to */
} tqp_dim;

typedef struct {
  int32_t src; /* 0 = fact column, 1 + d = column of dimension d */
  int32_t col; /* index into that table's columns */
} tqp_valref;

tqp_status tqp_star_agg(const tqp_col* fact_cols, int nfact_cols, int64_t n_fact,
                        const tqp_pred* fact_preds, int nfact_preds, const int* fk_col,
                        const tqp_dim* dims, int ndims, const tqp_valref* vals, int nvals,
                        const tqp_expr* exprs, int nexprs, const tqp_agg* aggs, int naggs,
                        void* const* d_out_keys, int64_t* d_out_aggs, int64_t cap,
                        int64_t* d_out_groups, void* ws, size_t* ws_bytes, tqp_stream_t stream);

/* ========================================================================
 * Learned range partitioner.
 *
 * The paper's third scenario (Section 3.3) runs a neural network inside the
 * same tensor program as the relational operators.  Here a small network is
 * trained, on the GPU, on the key distribution that the method's own sort
 * produces, and used to route rows into ordered key-range buckets before the
 * final sort, so that each bucket can be sorted on-chip.  Results never
 * depend on the model: any non-decreasing bucket function gives the same,
 * exact group-by.
 *
 * Model (TQP_CDF_HIDDEN = H hidden units, float32):
 *   key normalisation  q = (p - umin) >> shift   (p: order-preserving packed
 *                      key, q < 2^24 so the conversion is exact),
 *                      x = (float)q * inv;
 *   unit j             z_j = fmaf(w[j], x, b[j]), h_j = min(max(z_j, 0), 1);
 *   output             F = c, then F = fmaf(a[j], h_j, F) for j = 0..H-1;
 *   bucket of B        min(B - 1, (int)(min(max(F, 0), 1) * B)).
 * With w >= 0 and a >= 0 (kept by projection after every training step)
 * F and the bucket are non-decreasing in the key.
 * ====================================================================== */
#define TQP_CDF_HIDDEN 64

typedef struct {
  float w[TQP_CDF_HIDDEN];
  float b[TQP_CDF_HIDDEN];
  float a[TQP_CDF_HIDDEN];
  float c;
  int32_t shift;
  float inv;
  int32_t pad_;
  uint64_t umin;
} tqp_cdf_model; /* 792 bytes; lives in device memory */

typedef struct {
  int32_t epochs; /* full-sample Adam steps */
  float lr;       /* Adam (Kingma & Ba 2015) step size and moments */
  float beta1;
  float beta2;
  float eps;
  int32_t pad_;
} tqp_train_cfg;

/* tqp_cdf_forward: F[i] = model(x[i]) (float32, the fixed evaluation order
 * above) for i < n; if d_bucket is not NULL also its bucket of B.  d_F may
 * be NULL when d_bucket is given (the buckets alone are written). */
tqp_status tqp_cdf_forward(const tqp_cdf_model* d_model, const float* d_x, int64_t n, float* d_F,
                           int32_t* d_bucket, int B, tqp_stream_t stream);

/* tqp_cdf_backward: gradient of the mean-squared error
 * L = (1/n) sum_i (F(x_i) - y_i)^2 (F without the output clamp) with respect
 * to w, b, a, c: d_grad[0..H) = dL/dw, [H..2H) = dL/db, [2H..3H) = dL/da,
 * [3H] = dL/dc, [3H+1] = L.  Where a unit is clamped (z <= 0 or z >= 1) its
 * w and b receive no gradient.  Deterministic: fixed reduction order.
 * n <= 2^20. */
tqp_status tqp_cdf_backward(const tqp_cdf_model* d_model, const float* d_x, const float* d_y, int64_t n,
                            float* d_grad, void* ws, size_t* ws_bytes, tqp_stream_t stream);

/* tqp_cdf_train: cfg->epochs Adam steps on (x, y) starting from *d_model
 * (updated in place), each followed by the projection w, a >= 0.  The loss
 * before each step goes to d_loss[epoch] when d_loss is not NULL. n <= 2^20. */
tqp_status tqp_cdf_train(const float* d_x, const float* d_y, int64_t n, tqp_cdf_model* d_model,
                         const tqp_train_cfg* cfg, float* d_loss, void* ws, size_t* ws_bytes,
                         tqp_stream_t stream);

typedef struct {
  int32_t sample;  /* keys sampled (strided) to train on; power of two in [1024, 2^20].
                      Heavy keys are found in a strided sample 4 times larger (at
                      most 2^20 keys), whose every 4th sorted key is trained on. */
  int32_t buckets; /* learned buckets B (power of two <= 2^17); 0 = from n */
  int32_t train;   /* 1 = train the network; 0 = keep the identity CDF F(x) = x */
  int32_t heavy;   /* 1 = aggregate the sample's frequent keys directly */
  tqp_train_cfg train_cfg;
  int32_t init;    /* network before training: 0 = identity CDF, 1 = knots at the
                      sample's 1/H quantiles (the piecewise-linear empirical CDF) */
  int32_t pad_;
} tqp_learned_cfg;

typedef struct {          /* written to device memory by the learned group-by */
  int64_t buckets;        /* B */
  int64_t heavy_keys;     /* keys aggregated directly */
  int64_t light_rows;     /* rows routed through the buckets */
  int64_t max_bucket;     /* largest bucket (rows) */
  int64_t over_capacity;  /* buckets sorted by the global-memory fallback */
  int64_t nonempty;       /* non-empty buckets */
  int64_t over_capacity_rows; /* rows in buckets sorted by the fallback */
  int64_t small_rows;     /* rows in buckets of 2..1024 rows (sorted by one warp
                             when the bucket's key span is below 2^48) */
  float loss_first;       /* training loss of the network before training */
  float loss_last;        /* training loss of the returned network: training keeps the
                             parameters of the lowest loss it evaluated, so
                             loss_last <= loss_first */
} tqp_learned_stats;

/* ------------------------------------------------------------------------
 * tqp_groupby_agg_learned -- the group-by of tqp_groupby_agg (same inputs,
 * outputs and guarantees: bit-identical results) computed through the
 * learned range partitioner: key range and packing; a strided sample of the
 * packed keys sorted by the radix sort; empirical-CDF targets
 * (first rank + count / 2) / S per distinct sample key; GPU training; keys
 * that are frequent in the sample aggregated directly; the other rows
 * scattered into the network's buckets and each bucket sorted on-chip (a
 * bucket beyond the on-chip capacity is radix-sorted by one block in global
 * memory); one reduce-by-key over the sorted rows that merges the directly
 * aggregated keys in key order.  d_model_out (nullable) receives the trained
 * model, d_stats (nullable) the statistics above.
 * ---------------------------------------------------------------------- */
tqp_status tqp_groupby_agg_learned(const tqp_col* keys, int nkeys, const tqp_col* vals, int nvals,
                                   const tqp_expr* exprs, int nexprs, const tqp_agg* aggs, int naggs,
                                   const int32_t* d_sel, int64_t n, const int64_t* d_n,
                                   void* const* d_out_keys, int64_t* d_out_aggs, int64_t cap,
                                   int64_t* d_out_groups, const tqp_learned_cfg* cfg,
                                   tqp_cdf_model* d_model_out, tqp_learned_stats* d_stats, void* ws,
                                   size_t* ws_bytes, tqp_stream_t stream);

/* ------------------------------------------------------------------------
 * tqp_partition_learned -- the learned range partitioner on its own: the
 * rows (d_sel[0..n) or 0..n-1; n or *d_n) split into B ordered key-range
 * buckets by the network of this header's model, fit on the GPU to the
 * key distribution (the same fit as tqp_groupby_agg_learned: key range and
 * packing; a strided sample of SH = min(4 * cfg->sample, 2^20) packed keys,
 * sorted; with cfg->heavy, the sample's heavy keys -- counts of at least
 * max(2, floor(SH * 8192 / (2 n)) + 1), the most frequent ones, at most
 * 1024 -- set apart; training pairs on the CDF of the other (light) sample
 * keys from every (SH / sample)-th sorted key: x = the normalised key, y =
 * (light keys before it + half its light count) / light total; knots and
 * Adam training).  Outputs (each pointer may be NULL):
 *   d_bucket[i]   bucket id of the i-th row: a light row's bucket 0..B-1
 *                 (non-decreasing in the key), a row of heavy key h
 *                 (heavy keys ascending) the id B + h;
 *   d_rows[k]     the rows' ids grouped by bucket id, in input order within
 *                 a bucket (a stable counting sort by bucket id);
 *   d_offsets[b]  the first position of bucket id b in d_rows,
 *                 b = 0..B + 1024 (B + 1025 entries; the last ones n);
 *   d_train_x, d_train_y  the cfg->sample training pairs (float32);
 *   d_model_out   the trained network;  d_stats  the statistics below.
 * B = cfg->buckets, or (0) the power of two giving about 512 rows a bucket.
 * Two-phase workspace sizing; limits and errors as tqp_groupby_agg_learned.
 * ---------------------------------------------------------------------- */
#define TQP_MAX_HEAVY 1024
tqp_status tqp_partition_learned(const tqp_col* keys, int nkeys, const int32_t* d_sel, int64_t n, const int64_t* d_n,
                                 const tqp_learned_cfg* cfg, int32_t* d_bucket, int32_t* d_rows, int64_t* d_offsets,
                                 float* d_train_x, float* d_train_y, tqp_cdf_model* d_model_out,
                                 tqp_learned_stats* d_stats, void* ws, size_t* ws_bytes, tqp_stream_t stream);

/* ------------------------------------------------------------------------
 * tqp_star_agg_learned -- tqp_star_agg (same inputs, outputs, guarantees
 * and results) whose dimensions of at least 2^20 passing-row candidates
 * have their keys sorted through the learned range partitioner instead of
 * the radix sort: a strided sample of the keys sorted, the network fit to
 * its CDF (cfg: sample size, bucket count (0: 4096 to 8192 keys per bucket),
 * training, knots; heavy keys do not apply to unique keys), every key
 * placed in its bucket and every bucket sorted on chip.  The dimension keys
 * must be unique among the passing rows, as for tqp_star_agg.
 * ---------------------------------------------------------------------- */
tqp_status tqp_star_agg_learned(const tqp_col* fact_cols, int nfact_cols, int64_t n_fact,
                                const tqp_pred* fact_preds, int nfact_preds, const int* fk_col,
                                const tqp_dim* dims, int ndims, const tqp_valref* vals, int nvals,
                                const tqp_expr* exprs, int nexprs, const tqp_agg* aggs, int naggs,
                                void* const* d_out_keys, int64_t* d_out_aggs, int64_t cap,
                                int64_t* d_out_groups, const tqp_learned_cfg* cfg, void* ws,
                                size_t* ws_bytes, tqp_stream_t stream);

/* ========================================================================
 * Batched instances: many independent join + filter + group-by problems of
 * uneven size (the Q14 shape of Section 2.3, one query per problem) in one
 * sequence of persistent launches instead of one call per problem.
 *
 * Every problem has the same query shape (tqp_batch_shape):
 *   SELECT dim.group, aggs FROM fact JOIN dim ON fact.fk = dim.key
 *   WHERE fact predicates GROUP BY dim.group
 * with its own columns and sizes (tqp_problem).  All dimensions are sorted
 * by (problem, key) in one radix sort and grouped by (problem, group) in a
 * second; one persistent probe kernel pulls fact tiles of all problems from
 * one work queue (a tile never spans two problems) and folds each row into
 * its problem's group slots in shared memory; a final kernel writes each
 * problem's groups in ascending group order.  Dimension keys must be unique
 * within a problem (TQP_ERR_UNSUPPORTED on the device otherwise).
 * ====================================================================== */
#define TQP_BATCH_MAX_COLS 4

typedef struct {
  int32_t nfact_cols;
  int32_t fact_dtype[TQP_BATCH_MAX_COLS]; /* dtypes of the fact columns */
  int32_t fk_col;                         /* fact column holding the foreign key */
  int32_t key_dtype;                      /* TQP_I32 (dimension key and fact fk) */
  int32_t group_dtype;                    /* TQP_I8 / TQP_I16 / TQP_I32 */
  int32_t npred;
  tqp_pred preds[TQP_MAX_PREDS];          /* over fact columns; literals shared */
  int32_t nexprs;
  tqp_expr exprs[TQP_MAX_EXPRS];          /* terms index fact columns */
  int32_t naggs;
  tqp_agg aggs[TQP_MAX_AGGS];
} tqp_batch_shape;

typedef struct {
  int64_t n_fact;
  const void* fact_cols[TQP_BATCH_MAX_COLS]; /* device */
  int64_t n_dim;
  const void* dim_key;                       /* device, unique keys */
  const void* dim_group;                     /* device */
  void* out_keys;                            /* device, group_dtype, capacity cap */
  int64_t* out_aggs;                         /* device, [cap][naggs] */
  int64_t cap;
  int64_t* d_out_groups;                     /* device */
} tqp_problem;

typedef struct {
  int32_t probe_items; /* fact rows per thread per probe tile: 4, 8 or 16 (0 = 8) */
  int32_t pad_;
} tqp_batch_cfg;

/* tqp_star_agg_batched: runs all nprob problems (host array of
 * descriptors; device pointers inside).  Results per problem as for
 * tqp_star_agg.  Limits: nprob <= 65536, sum of n_dim < 2^30, each
 * problem's distinct group values <= 4096. */
tqp_status tqp_star_agg_batched(const tqp_batch_shape* shape, const tqp_problem* probs, int nprob,
                                const tqp_batch_cfg* cfg, void* ws, size_t* ws_bytes,
                                tqp_stream_t stream);

/* ------------------------------------------------------------------------
 * Device status and test hooks.
 * tqp_status_poll: synchronises `stream`, returns the current device's status
 * word (TQP_OK if no device-side error was recorded since the last poll) and
 * clears it.
 * tqp_debug_set_spin_limit: bound of every inter-block wait, in polling
 * rounds (default 1<<20, about a second); a wait that runs out records
 * TQP_ERR_TIMEOUT and the block gives up without writing results.
 * tqp_debug_inject_unpublished_tile: testing hook -- the scan tile with this
 * id (of the next launches) never publishes its status, so its successors'
 * bounded waits run out; -1 disables it.
 * ---------------------------------------------------------------------- */
tqp_status tqp_status_poll(tqp_stream_t stream);
/* tqp_sort_tiles: rows per thread of the radix sort's tiles (of 256
 * threads), process-wide, for 32-bit keys (8, 12 or 16; default 16) and
 * 64-bit keys (6, 8 or 12; default 12); 0 leaves a width unchanged.  Any
 * choice sorts identically; it only changes speed (the autotuner's knob).
 * A call's workspace is sized with the setting at its size query, so change
 * it between calls, not between a call's size query and the call. */
tqp_status tqp_sort_tiles(int items32, int items64);
tqp_status tqp_debug_set_spin_limit(int64_t rounds);
tqp_status tqp_debug_inject_unpublished_tile(int64_t tile);
const char* tqp_status_string(tqp_status s);

/* Instrumentation (no counterpart in the paper).
 * tqp_debug_launch_count: number of kernels this library has launched in
 * this process (host-side count of launch calls; a launch captured into a
 * CUDA graph counts once, at capture).
 * tqp_profile_events: from now on, record `start_event` just before and
 * `stop_event` just after the kernel(s) of one class, on the call's stream
 * (cudaEvent_t handles passed as void*; NULL clears).  Classes: 1 = fused
 * star probe, 2 = radix sort passes (from the first to the last pass of a
 * sort), 3 = filter, 4 = group-by reduce, 5 = join probe, 6 = batched probe,
 * 7 = learned bucket sort (block kernel), 8 = learned partition scatter,
 * 9 = learned bucket sort (warp kernel), 10 = network forward
 * (tqp_cdf_forward), 11 = string codes (all of tqp_string_codes), 12 / 13 =
 * the key sort (radix or learned, with its dense-key check) of star dimension
 * 0 / 1, 14 / 15 = the directory and cell records of star dimension 0 / 1.
 * Records are
 * external, so under stream capture they become event nodes of the graph. */
int64_t tqp_debug_launch_count(void);
tqp_status tqp_profile_events(int kernel_class, void* start_event, void* stop_event);

#ifdef __cplusplus
}
#endif

#endif /* TQP_H_ */
