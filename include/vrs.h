/*
 * vrs.h -- C ABI of the GB300 exact filtered vector search library.
 *
 * The library implements the exhaustive, scan-based access path for mixed
 * vector-relational search of Sanca & Ailamaki, "Efficient Data Access Paths
 * for Mixed Vector-Relational Search" (arXiv 2403.15807):
 *
 *   Sec. 3, eq. "Brute force similarity search with relational predicate":
 *       sigma_{eps, v, theta_R}(R) = sigma_eps(v x sigma_{theta_R}(R))
 *
 * i.e. a relational predicate theta_R on int32 attribute columns selects
 * rows (Sec. 3.2, predicate pushdown), a distance eps is evaluated between a
 * batch of query vectors and every selected row (Sec. 3.1, the batched
 * "Tensor formulation" for N:N, the per-tuple scan for 1:N / N:1), and the
 * k best rows per query are returned (top-k retrieval, Sec. 2.2 and Sec. 5).
 *
 * Conventions shared by every call:
 *  - Every call returns a vrs_status and never aborts.  On failure the
 *    thread-local message from vrs_last_error() says why.
 *  - Row ids are load positions 0..n-1.  Bitmaps are uint32 words; row i is
 *    bit (i % 32) of word (i / 32); bits past n are zero.
 *  - Predicates are conjunctions of half-open ranges lo <= attr[col] < hi; a
 *    predicate with 0 terms selects every row.
 *  - L2 results are squared Euclidean distances; IP results are q.x and rank
 *    larger-first.  Ties rank the smaller row id first.  When fewer than k
 *    rows qualify, the tail is padded with id -1 and distance +inf.
 *  - "on_device" flags say whether a pointer is device memory of the
 *    engine's GPU (1) or host memory (0).  Host buffers may be pageable.
 *  - A call that takes a stream (a cudaStream_t passed as void*, NULL = the
 *    legacy default stream) enqueues its GPU work on it.  When every
 *    input and output is in device memory the call returns without waiting
 *    for the GPU; otherwise it synchronises the stream before returning.
 *  - The caller owns every buffer it passes.  The engine copies vectors and
 *    attributes into device memory it owns and frees in vrs_destroy; it also
 *    owns a growable device workspace reused across queries.  Calls on one
 *    engine must not run concurrently from several host threads.
 */
#ifndef VRS_H
#define VRS_H

#include <stdint.h>

#if defined(__GNUC__)
#define VRS_API __attribute__((visibility("default")))
#else
#define VRS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vrs_engine vrs_engine; /* opaque; owned by the library */

typedef enum {
    VRS_OK = 0,
    VRS_EINVAL = -1,   /* bad argument (null pointer, size, column, k ...) */
    VRS_ENOMEM = -2,   /* device or host allocation failed */
    VRS_ECUDA = -3,    /* a CUDA call failed; the message names it */
    VRS_ETIMEOUT = -4, /* a bounded device-side wait ran out */
    VRS_ESTATE = -5,   /* call out of order (e.g. query before load) */
    VRS_EIO = -6,      /* file could not be read or is malformed */
    VRS_EINTERNAL = -7, /* a device-side capacity invariant failed (a candidate
                          list would have overflowed); results are invalid */
    VRS_ESIZE = -8     /* an output capacity is too small; the size needed is
                          reported (vrs_range_query) */
} vrs_status;

typedef enum { VRS_L2 = 0, VRS_IP = 1 } vrs_metric;

/* Storage / arithmetic types.  Used as values and as bit positions in the
 * copies mask of vrs_load_vectors (1u << VRS_F32 ...). */
typedef enum { VRS_F32 = 0, VRS_BF16 = 1, VRS_FP8E4M3 = 2 } vrs_dtype;

/* One term lo <= attr[col][row] < hi of a conjunction (Sec. 3.2). */
typedef struct {
    int32_t col;
    int32_t lo;
    int32_t hi;
} vrs_range;

/* Conjunction of n_terms ranges; n_terms == 0 selects every row. */
typedef struct {
    int32_t n_terms;
    const vrs_range *terms;
} vrs_pred;

/* Scan plans: how the distance stage visits the selected rows.
 *  GEMV          per-tuple scan (1:N / N:1, Sec. 3.1) over the compacted
 *                ids with float32 operands: on the tensor cores (float32
 *                split into exactly representable parts, see
 *                VRS_OPT_TENSOR_GEMV) for up to 64 queries, else FP32 FMAs
 *                on the CUDA cores;
 *  COMPACT_GEMM  predicate first, then the batched tensor formulation over
 *                the gathered qualifying rows (late materialisation,
 *                Sec. 3.2 / Fig. 3), on tensor cores;
 *  MASK_GEMM     tensor formulation over every row with the predicate
 *                applied on the fly to the scores (Sec. 3.2, first strategy). */
enum {
    VRS_PLAN_AUTO = -1,
    VRS_PLAN_GEMV = 0,
    VRS_PLAN_COMPACT_GEMM = 1,
    VRS_PLAN_MASK_GEMM = 2,
    VRS_PLAN_CELLS = 3   /* batches of per-query ranges over a grid (vrs_build_grid) */
};

/* Engine options (vrs_set_option). */
enum {
    VRS_OPT_KPRIME_FACTOR = 0, /* candidates kept before re-rank:
                                  k' = max(f*k, k + 8, 8*f) with f = this factor
                                  (0 = default: 2 for F32, 4 for BF16, 16 for FP8);
                                  batched launches apply it per query.  It
                                  changes speed only: a query whose k' was too
                                  small is widened until certified exact */
    VRS_OPT_RERANK = 1,        /* 1 (default): exact FP32 re-rank of the k'
                                  candidates; 0: return the first-pass scores */
    VRS_OPT_GRID_CTAS = 2,     /* 0 (default): automatic; else CTAs per query
                                  group for the distance kernels */
    VRS_OPT_PROFILE = 3,       /* 1: record CUDA events around every stage of
                                  each query (read with vrs_last_profile) */
    VRS_OPT_FUSED_SCAN = 4,    /* 1: the GEMV plan evaluates the predicate on
                                  the fly inside the distance kernel (Sec. 3.2,
                                  first strategy); 0 (default): predicate,
                                  compaction and distance run as separate
                                  kernels (predicate-first) */
    VRS_OPT_BATCHED = 5,       /* 1 (default): a batch with one predicate per
                                  query and BF16/FP8 compute runs as one
                                  launch of the tensor kernel with each query's
                                  conjunction applied to its own scores (up to
                                  4 distinct columns); 0: one pass per query */
    VRS_OPT_GRAPH = 6,         /* 1 (default): the batched launch's kernel
                                  sequence is captured once per shape into a
                                  CUDA graph and replayed */
    VRS_OPT_TMA = 7,           /* 1 (default): tensor-core plans load query
                                  tiles and dense row tiles with TMA; 0: with
                                  cp.async 16-byte copies */
    VRS_OPT_DENSE_KEYS = 8,    /* 1 (default): GEMV batches whose key matrix
                                  (batch x rows x 4 B) fits 256 MB write every
                                  first-pass key and each query's minimum per
                                  128 positions; the merge bounds the k'-th key
                                  by the k'-th smallest of up to 4k' chunk-group
                                  minima, reads only the chunks at or below it
                                  and selects the k' best exactly; 0: select
                                  inside the scan */
    VRS_OPT_SELECT_CAP = 9,    /* capacity of that merge's list (chunk minima,
                                  then the candidate keys) per query (0,
                                  default: room for the minima of the selection
                                  and 4k', at least 4096), at most what fits
                                  the CTA's shared memory; a query whose candidates
                                  overflow is selected from its whole key row,
                                  so any value gives the same results */
    VRS_OPT_STAGED_SCAN = 10,  /* 1: the CUDA-core dense-key GEMV distance pass
                                  stages rows in shared memory with bulk
                                  asynchronous copies (one CTA per SM) when a
                                  few stages of 128 rows fit; 0 (default):
                                  rows are read straight into registers */
    VRS_OPT_TENSOR_GEMV = 11,  /* 1 (default): the dense-key GEMV distance pass
                                  over float32 rows runs on the tensor cores
                                  (128 rows x up to 64 queries per MMA, three
                                  products per pair, FP32 accumulation): over
                                  the bf16 pair copy (VRS_OPT_PAIR_COPY), else
                                  float32 split into TF32 high and low parts;
                                  0: on the CUDA cores */
    VRS_OPT_CERT_SAMPLE = 15,  /* 1 (default): a tensor plan over a lossy
                                  encoding (BF16 or E4M3 rows of a float32
                                  table) first runs about 1/16 of the selected
                                  rows with an exact re-rank; their k-th exact
                                  distance D bounds the selection's, so one
                                  full pass seeded at D + E (the certificate's
                                  bound) keeps every row the exact top-k can
                                  hold.  0: a full first pass of width k', and
                                  a seeded full pass only for queries it could
                                  not certify.  With 1, an E4M3 request on a
                                  tensor plan runs on the BF16 copy when one is
                                  resident: E4M3's error band is too wide for
                                  any affordable pass width */
    VRS_OPT_WAIT_TEST = 14,    /* test hook, one-shot: 1 makes the next
                                  tensor-core GEMV pass over the pair copy wait
                                  on a barrier nothing arrives at; the bounded
                                  wait gives up after ~1 s, the kernel aborts
                                  and drains, and the call returns
                                  VRS_ETIMEOUT (when it synchronises; else the
                                  next synchronising call does) with the
                                  engine left usable */
    VRS_OPT_PAIR_COPY = 13,    /* 1 (default): vrs_load_vectors also keeps a
                                  bf16 pair copy of the float32 rows (x1 =
                                  bf16(x), x2 = bf16(x - x1); the same 4 bytes
                                  per element), and the tensor-core GEMV pass
                                  reads it with bf16 MMAs (q1.x1 + q1.x2 +
                                  q2.x1) instead of splitting float32 rows into
                                  TF32 parts at query time; set it before
                                  loading.  0: no pair copy */
    VRS_OPT_ZERO_COPY = 17,    /* 1 (default): a host-buffer vrs_query on the
                                  captured GEMV form whose queries and outputs
                                  are page-locked reads and writes them in
                                  place from the kernels (their device
                                  addresses; over NVLink-C2C on Grace
                                  machines), with no copies; 0: copies to and
                                  from device buffers inside the same graph */
    VRS_OPT_CELL_PLAN = 16,    /* 1 (default): a batch whose per-query
                                  predicates are ranges on the two columns of
                                  the grid vrs_build_grid made runs the cell
                                  plan (BF16 compute); 0: the batched mask
                                  plan */
    VRS_OPT_SEED_BOUND = 12    /* 1 (default): BF16 MASK_GEMM with at least
                                  8192 selected rows per CTA, and E4M3 on
                                  either tensor plan from 2048, first runs
                                  evenly spaced selected rows (about 1/16 of
                                  the selection) through the same kernel and
                                  starts every query's bound one past their
                                  k'-th best first-pass key, so the full pass
                                  inserts few keys into its heaps (same
                                  results); 0: no sample pass */
};

/* Query stages timed when VRS_OPT_PROFILE is on (the breakdown of Fig. 6:
 * filtering, materialisation, computation). */
enum {
    VRS_STAGE_PREPARE = 0,   /* query upload / padding */
    VRS_STAGE_PREDICATE = 1, /* theta_R -> bitmap + tile counts */
    VRS_STAGE_OFFSETS = 2,   /* tile counts -> offsets, total */
    VRS_STAGE_COMPACT = 3,   /* bitmap -> ascending ids */
    VRS_STAGE_DISTANCE = 4,  /* distance pass (+ per-CTA top-k' when fused) */
    VRS_STAGE_MERGE = 5,     /* selection of the k' best, exact re-rank,
                                final top-k */
    VRS_N_STAGES = 6
};

/* Library version as "major.minor.patch". */
VRS_API const char *vrs_version(void);

/* Thread-local text of the last error on this thread ("" if none). */
VRS_API const char *vrs_last_error(void);

/* Create an engine on CUDA device `device`.  *out receives the handle.  The
 * learned plan model shipped next to the library (data/planner_gb300.bin in
 * the library's directory; environment variable VRS_PLANNER names another
 * file, or "none") is loaded as by vrs_planner_load; when it is missing or
 * invalid the engine keeps the fixed rule, and vrs_create still succeeds.
 * Errors: EINVAL (null out, bad device), ECUDA, ENOMEM. */
VRS_API vrs_status vrs_create(int device, vrs_engine **out);

/* Free every device buffer the engine owns and the engine itself.  Waits for
 * the engine's outstanding work.  NULL is accepted (no-op). */
VRS_API vrs_status vrs_destroy(vrs_engine *eng);

/* Load the vector column of table R (Sec. 3: column store of vector and
 * relational columns).  x is [n x d] row-major: float32 values when
 * in_dtype == VRS_F32, bfloat16 bit patterns (uint16) when VRS_BF16.
 * copies: mask of (1u << dtype) resident encodings to build:
 *   F32   float32 copy (the "master" used for exact re-rank);
 *   BF16  bfloat16 copy, round-to-nearest-even of the input;
 *   FP8   E4M3 copy with one float32 scale per row, scale = max|x|/448.
 * For in_dtype == BF16 the stored values are the bf16 input itself and the
 * re-rank reads them (the F32 bit may still be set to keep a widened copy).
 * Also computes ||x_i||^2 per row in float32 with compensated summation.
 * Replaces any previous vectors (attributes must then be reloaded with the
 * same n).  Errors: EINVAL (n < 1, d < 1, d > 4096, bad mask), ENOMEM, ECUDA. */
VRS_API vrs_status vrs_load_vectors(vrs_engine *eng, const void *x, int64_t n, int32_t d,
                            vrs_dtype in_dtype, uint32_t copies, int x_on_device,
                            void *stream);

/* Load relational column `col` (0 <= col < 8): int32 [n], n equal to the
 * vector count.  Errors: EINVAL, ESTATE (no vectors), ENOMEM, ECUDA. */
VRS_API vrs_status vrs_load_attribute(vrs_engine *eng, int32_t col, const int32_t *a, int64_t n,
                              int a_on_device, void *stream);

/* Order-preserving int32 image of a float attribute value (richer predicates,
 * Table 1 "Any Expression": float columns through the same range stage).
 * For floats a < b (not NaN) key(a) < key(b); -0 and +0 map to 0; every NaN
 * maps to INT32_MAX, which no half-open range [lo, hi) contains.  So
 * lo <= a < hi on a float column is the int32 range [key(lo), key(hi)), and
 * lo <= a <= hi is [key(lo), key(hi) + 1).  Host function; no errors. */
VRS_API int32_t vrs_float_key(float v);

/* Load float32 attribute column `col` as its vrs_float_key image (host
 * conversion; a device array is copied to the host first), so predicates on
 * it use the int32 ranges above.  Errors as vrs_load_attribute. */
VRS_API vrs_status vrs_load_attribute_f32(vrs_engine *eng, int32_t col, const float *a, int64_t n,
                                          int a_on_device, void *stream);

/* Two-column grid for batches of per-query ranges (the cell plan; the
 * batched N:N Tensor formulation of Sec. 3.1 with each query's own predicate
 * of Sec. 3.2).  The values of columns col0 and col1 (both loaded) are cut
 * at quantiles of a sample of each column into `bins` bins (0: about
 * sqrt(n / 2048), at most 64; repeated values give fewer); every row falls
 * into one cell (its bin of each column), and the engine keeps a clustered
 * copy of the table -- bf16 rows, norms, the two columns, original ids --
 * stored cell by cell (n * (2 max(ld, 64) + 16) bytes; ld = d rounded up to
 * 16).  Afterwards
 * a vrs_query with one predicate per query whose terms are all on col0 and
 * col1, with compute VRS_BF16, reads for each query only the cells its
 * ranges overlap (VRS_PLAN_CELLS, unless VRS_OPT_CELL_PLAN is 0); results
 * are certified exact like every vrs_query.  Reloading the vectors or
 * either column drops the grid.  Needs the bf16 copy and d <= 256.  The
 * call synchronises `stream`.  Errors: EINVAL (columns, bins, d), ESTATE
 * (no vectors, a column not loaded, no bf16 copy), ENOMEM, ECUDA. */
VRS_API vrs_status vrs_build_grid(vrs_engine *eng, int32_t col0, int32_t col1, int32_t bins,
                                  void *stream);

/*
 * Filtered exact top-k for a batch of queries (Sec. 3 eq. with predicate
 * pushdown; top-k as in Sec. 5 "Vector Index").
 *   q        [batch x d] float32, row-major (device if io_on_device)
 *   preds    host array of n_preds predicates: n_preds == 1 shares one
 *            predicate across the batch, n_preds == batch gives one each
 *   k        host array of n_k values, n_k == 1 or batch; 0 <= k <= k_max
 *   k_max    row stride of the outputs, 1 <= k_max <= 256
 *   metric   VRS_L2 or VRS_IP (cosine = IP on normalised vectors, Sec. 3.1)
 *   compute  encoding the first distance pass reads (must be resident);
 *            the k' best first-pass candidates are then re-ranked exactly
 *            in FP32 from the highest-precision resident copy
 *   out_ids  [batch x k_max] int64 (device if io_on_device)
 *   out_dist [batch x k_max] float32 (device if io_on_device)
 * Exactness: every query is certified before it is returned.  With D the
 * k-th exact distance among the k' re-ranked candidates and E a worst-case
 * bound on the first pass's error for that query (Cauchy-Schwarz over the
 * encoding residuals measured at load and at query preparation, plus the
 * products' FP32 accumulation), the result is exact once D stays below the
 * k'-th first-pass key minus E.  A query that fails the test is run again:
 * the dense-key GEMV merge re-ranks every row whose first-pass key is within
 * D + E itself; other plans re-run the query as part of a sub-batch, first
 * as a wider tensor pass (BF16 when resident) that keeps every row within
 * D + E, then through the dense-key GEMV plan.  vrs_last_cert reports how.
 * With io_on_device the call is asynchronous on `stream` (NULL: the legacy
 * default stream) when every first pass ran the dense-key GEMV form; the
 * tensor plans and the in-scan GEMV selection synchronise the stream once to
 * read their certificates.  Otherwise the call returns after the results are
 * in the host buffers, and without a stream it runs on a stream the engine
 * owns.
 * Errors: EINVAL, ESTATE (vectors or a used column not loaded), ENOMEM,
 * ECUDA, ETIMEOUT, EINTERNAL (a query could not be certified: the dense-key
 * form does not fit, n * 4 bytes above 256 MB).
 */
VRS_API vrs_status vrs_query(vrs_engine *eng, const float *q, int32_t batch, int32_t d,
                     const vrs_pred *preds, int32_t n_preds, const int32_t *k, int32_t n_k,
                     int32_t k_max, vrs_metric metric, vrs_dtype compute, int64_t *out_ids,
                     float *out_dist, int io_on_device, void *stream);

/* Filtered range search: the selection sigma_eps of Sec. 3 (eq. "Brute force
 * similarity search with relational predicate theta"), with eps a bound on
 * the score, over the rows one shared predicate selects.  Query i keeps every
 * selected row whose squared L2 distance is <= eps (VRS_L2), or whose q.x is
 * >= eps (VRS_IP).  Scores are exact FP32 (the direct forms sum (q-x)^2 and
 * sum q x over the float32 copy), so a row whose score lies within FP32
 * rounding of eps may fall on either side.
 *   q           [batch x d] float32 (host, or device when io_on_device)
 *   batch       1..64; the key matrix [batch x rows] float32 must fit 256 MB
 *   pred        one predicate for the whole batch
 *   out_offsets [batch + 1] int64, host memory, always written: query i's
 *               results are out_ids / out_dist [out_offsets[i], out_offsets[i+1])
 *               (in no particular order)
 *   out_ids     [cap] int64 row ids; out_dist [cap] float32 scores (squared
 *               distance, or q.x); host or device memory per io_on_device
 * The call synchronises with its stream (the result count decides the
 * output).  When the results exceed cap, only out_offsets is written and
 * VRS_ESIZE is returned: call again with cap >= out_offsets[batch].
 * Requires the float32 copy.  Errors: EINVAL, ESTATE, ESIZE, ENOMEM, ECUDA,
 * ETIMEOUT. */
VRS_API vrs_status vrs_range_query(vrs_engine *eng, const float *q, int32_t batch, int32_t d,
                                   const vrs_pred *pred, float eps, vrs_metric metric,
                                   int64_t cap, int64_t *out_offsets, int64_t *out_ids,
                                   float *out_dist, int io_on_device, void *stream);

/* Top-k under a disjunction of conjunctions (richer predicates, Table 1 "Any
 * Expression"): a row qualifies when any of the n_conj conjunctions holds;
 * an IN-list on one column is n_conj one-term conjunctions [v, v + 1).  The
 * query path runs once per conjunction and the k best of the union of those
 * lists are kept, each row once (exact: the union's k best are each among
 * its own conjunction's k best).  One k for the batch; n_conj * k <= 2048.
 * q, out_ids [batch x k], out_dist [batch x k] as in vrs_query (padding -1 /
 * +inf).  Errors: EINVAL, ESTATE, ENOMEM, ECUDA, ETIMEOUT. */
VRS_API vrs_status vrs_query_dnf(vrs_engine *eng, const float *q, int32_t batch, int32_t d,
                                 const vrs_pred *conj, int32_t n_conj, int32_t k,
                                 vrs_metric metric, vrs_dtype compute, int64_t *out_ids,
                                 float *out_dist, int io_on_device, void *stream);

/* Vector join: batched queries drawn from a relation (the N:N tensor form of
 * Sec. 3.1 with the query side a relation of its own).  The query relation
 * Q (m rows of d float32 values, with q_cols int32 attribute columns) is
 * filtered by qpred; each selected query row gets the exact filtered top-k
 * of the loaded rows that rpred selects, as vrs_query computes it.
 *   qrel        [m x d] float32; qattrs [q_cols x m] int32 (may be NULL when
 *               q_cols == 0); host or device memory per io_on_device
 *   qpred       conjunction over Q's columns 0..q_cols-1; rpred over the
 *               loaded attribute columns
 *   *out_nq     (host) number of selected query rows, always written
 *   out_qids    [cap] int64, host memory: the selected query rows, ascending
 *   out_ids / out_dist  [cap x k]: row j holds the top-k of query row
 *               out_qids[j] (ids -1 and +inf past the selection), in host or
 *               device memory per io_on_device
 * The call synchronises with its stream.  When more than cap query rows are
 * selected only *out_nq is written and VRS_ESIZE is returned.  Errors:
 * EINVAL, ESTATE, ESIZE, ENOMEM, ECUDA, ETIMEOUT. */
VRS_API vrs_status vrs_join_topk(vrs_engine *eng, const float *qrel, int64_t m, int32_t d,
                                 const int32_t *qattrs, int32_t q_cols, const vrs_pred *qpred,
                                 const vrs_pred *rpred, int32_t k, vrs_metric metric,
                                 vrs_dtype compute, int64_t cap, int64_t *out_nq,
                                 int64_t *out_qids, int64_t *out_ids, float *out_dist,
                                 int io_on_device, void *stream);

/* Evaluate theta_R alone (Sec. 3.2, the filtering step): bitmap_out receives
 * ceil(n/32) uint32 words, *count_out (host) the number of selected rows.
 * bitmap_out may be NULL.  Errors: EINVAL, ESTATE, ENOMEM, ECUDA. */
VRS_API vrs_status vrs_eval_predicate(vrs_engine *eng, const vrs_pred *pred, uint32_t *bitmap_out,
                              int64_t *count_out, int out_on_device, void *stream);

/* Measurement hook, not part of the query path: read in full every row
 * ids[0..m) of the row-major device table `rows` (n_rows rows of row_bytes,
 * a multiple of 16; rows 16-byte aligned) and add the sum of what was read,
 * as floats, to the device float *out (which the caller zeroes); ids outside
 * [0, n_rows) are skipped.  This is the distance pass's access pattern over
 * a selection (each selected row read once) with no arithmetic to hide, so
 * its time bounds how fast any pass over those rows can be.  Asynchronous on
 * `stream` (NULL: the legacy default stream).  Errors: EINVAL, ECUDA. */
VRS_API vrs_status vrs_probe_gather(const void *rows, int64_t n_rows, int64_t row_bytes,
                                    const int32_t *ids, int64_t m, float *out, void *stream);

/* Late materialisation of the selection (Sec. 3.2, Fig. 3): ids_out receives
 * the ascending ids of the selected rows (capacity n int32), *count_out
 * (host) their number.  Errors: EINVAL, ESTATE, ENOMEM, ECUDA. */
VRS_API vrs_status vrs_select_ids(vrs_engine *eng, const vrs_pred *pred, int32_t *ids_out,
                          int64_t *count_out, int out_on_device, void *stream);

/* Copy out the per-row ||x||^2 (float32 [n]) the engine computed at load. */
VRS_API vrs_status vrs_get_norms(vrs_engine *eng, float *out, int out_on_device, void *stream);

/* Copy out a resident encoding: codes [n x d] (float32, bf16 bits or E4M3
 * bytes by dtype) and, for FP8, the per-row scales [n] (scale_out may be NULL
 * otherwise).  Errors: EINVAL, ESTATE (encoding not resident). */
VRS_API vrs_status vrs_get_encoded(vrs_engine *eng, vrs_dtype dtype, void *codes_out, float *scale_out,
                           int out_on_device, void *stream);

/* Force a scan plan (VRS_PLAN_*) for later queries; VRS_PLAN_AUTO (-1)
 * restores the planner.  Errors: EINVAL. */
VRS_API vrs_status vrs_set_plan(vrs_engine *eng, int plan);

/* Plan used by the last vrs_query (VRS_PLAN_*). */
VRS_API vrs_status vrs_last_plan(vrs_engine *eng, int *plan);

/* Set an engine option (VRS_OPT_*).  Errors: EINVAL. */
VRS_API vrs_status vrs_set_option(vrs_engine *eng, int key, int64_t value);

/* Timing of the last vrs_query run with VRS_OPT_PROFILE on: stage_ms
 * [VRS_N_STAGES] milliseconds per stage (summed over the query's passes,
 * from CUDA events on the query's stream; waits for them), *launches the
 * number of kernels the query launched, *selected the number of rows its
 * (last) predicate selected.  Any output pointer may be NULL.
 * Errors: EINVAL, ESTATE (profiling was off for the last query). */
VRS_API vrs_status vrs_last_profile(vrs_engine *eng, float *stage_ms, int32_t *launches,
                                    int64_t *selected);

/* Row-sharded search: a table split into contiguous row ranges, one engine
 * (one GPU) per range, every engine answering the same query batch.  Rows
 * are independent under the selection (Sec. 3, eq. "Brute force similarity
 * search with relational predicate": sigma filters rows one by one), so a
 * query's global top-k is the k best of the union of the shards' top-k
 * lists.  This merges them on the current device.
 *   ids, dist   [n_shards x batch x k]: shard s's vrs_query output (its local
 *               row ids, padding id -1 / +inf), shard-major
 *   row_offset  [n_shards] host int64: global id of shard s's row 0
 *   out_ids     [batch x k] global ids, out_dist [batch x k], in the
 *               vrs_query order and padding
 * 1 <= n_shards <= 64, n_shards * k <= 2048, global ids below 2^31.  With
 * io_on_device the four arrays are device memory and the call is
 * asynchronous on `stream`; otherwise they are host memory and the call
 * synchronises.  Errors: EINVAL, ECUDA. */
VRS_API vrs_status vrs_merge_shards(const int64_t *ids, const float *dist, int32_t n_shards,
                                    int32_t batch, int32_t k, const int64_t *row_offset,
                                    vrs_metric metric, int64_t *out_ids, float *out_dist,
                                    int io_on_device, void *stream);

/* How the queries of the last vrs_query, vrs_query_dnf or vrs_join_topk call
 * were certified exact (see vrs_query): counts[0] by their first pass,
 * counts[1] after the dense-key merge widened its candidates, counts[2] by
 * a wider tensor pass, counts[3] by the exact GEMV plan (a query of a
 * disjunction or join counts once per pass).  Waits for the last call's GPU
 * work.  Errors: EINVAL, ECUDA. */
VRS_API vrs_status vrs_last_cert(vrs_engine *eng, int64_t *counts);

/* First-pass kernel families for vrs_cert_bound: FP32 FMAs; float32 split
 * into TF32 parts (3 products); float32 split into two bf16 parts (3
 * products); bf16 operands; E4M3 operands with per-vector scales. */
enum { VRS_CERT_FFMA = 0, VRS_CERT_TF32X3 = 1, VRS_CERT_BF16X3 = 2, VRS_CERT_BF16 = 3,
       VRS_CERT_E4M3 = 4 };

/* The certificate's bound E on |first-pass key - exact key| (vrs_query) for
 * a query of norm qnorm whose encoding residual is qres, over rows of norm
 * at most xmax whose encoding residuals are at most xres, in dimension d.
 * Host function; returns -1 for an unknown kind or metric. */
VRS_API float vrs_cert_bound(int32_t kind, int32_t d, vrs_metric metric, float qnorm, float qres,
                             float xmax, float xres);

/* Load learned plan-model weights from `path` (the access-path choice the
 * paper leaves to an optimizer, Sec. 5.2/5.3 takeaways).  File format, all
 * little-endian: "VRSPLAN1", u32 version (1), u32 parameter count (4803),
 * f32 feature mean[6], f32 feature std[6], f32 output mean, f32 output std,
 * f32 parameters[4803] (layout of vrs_mlp_*), u64 FNV-1a checksum of every
 * preceding byte.  Features of a query: ln N, ln d, ln batch, ln selectivity
 * (sampled estimate, floor 1e-6), ln k, bytes per element of the compute
 * dtype; outputs: standardised ln(ms) of GEMV, COMPACT_GEMM, MASK_GEMM.  With
 * a model loaded and the plan not forced, each query takes the plan of
 * smallest predicted latency among the plans its compute dtype supports
 * (F32: GEMV; BF16: all three; FP8: the two tensor plans).  On any failure
 * (missing, truncated, bad magic, version or checksum) the engine keeps the
 * fixed rule and EIO is returned.  A NULL path unloads the model. */
VRS_API vrs_status vrs_planner_load(vrs_engine *eng, const char *path);

/* Plan-selection network 6 -> 64 -> 64 -> 3 (ReLU), on the current CUDA
 * device.  No counterpart in the paper (it names no cost model).  Parameters
 * are float32 W1[64x6] b1[64] W2[64x64] b2[64] W3[3x64] b3[3], row-major;
 * every array is host memory; X is [m x 6], T and mask are [m x 3].
 * vrs_mlp_forward: Y [m x 3]; bf16 != 0 rounds weights, inputs and
 *   activations to bf16 (float32 accumulation), the engine's inference form.
 * vrs_mlp_grad: gradient of loss = sum(mask*(Y-T)^2)/sum(mask) w.r.t. the
 *   parameters (grad [4803]) and the loss, float32.
 * vrs_mlp_train: `steps` full-batch Adam steps (beta 0.9/0.999, eps 1e-8) on
 *   params in place; *loss_out = loss at the returned parameters.
 * Errors: EINVAL (NULL, m < 1, all-zero mask), ECUDA, ENOMEM. */
VRS_API int32_t vrs_mlp_nparams(void);
VRS_API vrs_status vrs_mlp_forward(const float *params, const float *X, int64_t m, int32_t bf16,
                                   float *Y);
VRS_API vrs_status vrs_mlp_grad(const float *params, const float *X, const float *T,
                                const float *mask, int64_t m, float *grad, float *loss);
VRS_API vrs_status vrs_mlp_train(float *params, const float *X, const float *T, const float *mask,
                                 int64_t m, int32_t steps, float lr, float *loss_out);

/*
 * Filtered FP32 top-k without an engine and without device allocation.
 * No counterpart in the paper: this is for callers that cannot allocate
 * device memory while they run -- code inside a CUDA graph capture, hosts
 * whose allocator owns the whole pool, or services that fix their memory
 * budget at start-up.  It runs the GEMV plan's CUDA-core kernels on
 * caller-owned device buffers and keeps its working state in one fixed
 * device array of about 8.4 MB that every GPU loading the library holds
 * until exit.  Each call scans every row: it computes ||x||^2 of the whole
 * table (4 n d bytes read) and the distances of every row with the
 * predicate applied as a bitmap (another 4 n d bytes), so its cost grows
 * with n, not with the selection.
 *   x       [n x d] float32 rows, row-major, device memory
 *   attrs   [n_cols x n] int32 attribute columns, device, 16-byte aligned
 *           (n a multiple of 4 when n_cols > 1); x is 16-byte aligned too
 *   pred    host predicate on columns 0..n_cols-1
 *   q       [batch x d] float32 queries, device
 *   out_ids [batch x k] int64, out_dist [batch x k] float32, device
 *   status  optional device int32 (NULL: not written), set by the call's
 *           kernels: 0 every query's result is certified exact (the
 *           certificate of vrs_query); 1 a query's k'-candidate set could
 *           not be certified (its result is the exact re-rank of the
 *           first pass's candidates, which may miss a near-tied row); 2 a
 *           device-side invariant failed (results invalid).  Read it after
 *           synchronising the stream.
 * Limits: 1 <= n <= 2^20, d a multiple of 16 in 16..1024, 1 <= batch <= 32,
 * 1 <= k <= 64, 0 <= n_cols <= 8; larger sizes return VRS_EINVAL.
 * Asynchronous on `stream`; calls no cudaMalloc/cudaFree.  The first call on
 * a device looks up the array's device address (make it before any stream
 * capture).  Calls share the array: calls that overlap on the GPU race, so
 * serialise them.  Results follow the vrs_query conventions.
 */
VRS_API vrs_status vrs_query_noalloc(const float *x, int64_t n, int32_t d, const int32_t *attrs,
                                     int32_t n_cols, const vrs_pred *pred, const float *q,
                                     int32_t batch, int32_t k, vrs_metric metric,
                                     int64_t *out_ids, float *out_dist, int32_t *status,
                                     void *stream);

#ifdef __cplusplus
}
#endif

#endif /* VRS_H */
