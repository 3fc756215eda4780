// vrs_internal.cuh -- shared declarations of the library's kernels and
// device helpers.  Internal to the library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

namespace vrs {

constexpr int kMaxCols = 8;       // relational columns per engine
constexpr int kMaxTerms = 8;      // ranges per predicate
constexpr int kMaxK = 256;        // largest k per query
constexpr int kMaxKp = 1024;      // largest default candidate width k'
constexpr int kMaxKpWide = 4096;  // largest k' of a widened (certifying) pass
constexpr int kTileRows = 4096;   // rows per predicate/compaction tile (128 words)

// A predicate in kernel-argument form: conjunction of lo <= a[col] < hi.
struct PredArg {
    int32_t n_terms;
    int32_t col[kMaxTerms];
    int32_t lo[kMaxTerms];
    int32_t hi[kMaxTerms];
};

// Device pointers to the attribute columns.
struct AttrArg {
    const int32_t *col[kMaxCols];
};

// ---------------------------------------------------------------------------
// (key, id) composites.  A candidate is one uint64: the order-preserving
// uint32 image of its float key in the high half and the row id in the low
// half, so that ascending composite order is ascending key with ties broken
// by the smaller id, and composites of distinct rows never tie.
// ---------------------------------------------------------------------------
constexpr uint64_t kEmpty = ~0ull;

__host__ __device__ __forceinline__ uint32_t float_to_ordered(float f) {
#ifdef __CUDA_ARCH__
    uint32_t b = __float_as_uint(f);
#else
    uint32_t b;
    memcpy(&b, &f, 4);
#endif
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__host__ __device__ __forceinline__ float ordered_to_float(uint32_t u) {
    uint32_t b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    memcpy(&f, &b, 4);
    return f;
#endif
}

__device__ __forceinline__ uint64_t make_cand(float key, int32_t id) {
    return ((uint64_t)float_to_ordered(key) << 32) | (uint32_t)id;
}

// ---------------------------------------------------------------------------
// Exactness certificate of a first pass.
//
// The first pass ranks rows by an approximate key (reduced-precision operands,
// or FP32 operands split for the tensor core); the k' best are then re-ranked
// with the exact FP32 direct form.  Let E bound |first-pass key - exact key|
// for every row of the query.  With D the k-th exact key among the k'
// candidates (rounded up to cover the FP32 re-rank's own rounding) and kth'
// the k'-th first-pass key, every row outside the candidate set has an exact
// key >= kth' - E.  So when D < kth' - E the k best exact rows all lie among
// the candidates and the result is the exact top-k (up to FP32 rounding of
// the re-rank): the query is certified.  Otherwise every row that can still
// belong to the top-k has a first-pass key <= D + E, which bounds the rows a
// wider pass must examine.
//
// E (Cauchy-Schwarz on the encoding residuals, worst case over the rows):
//   dot error   <= |q| R + r (A + R) + P (|q| + r)(A + R)
//   L2: E = 2 dot error + (d + 32) u (|q|^2 + A^2)    (norm and key rounding)
//   IP: E =   dot error + (d + 32) u |q| A
// with A = max |x| over the re-rank copy, R = max |x - x_enc| over the rows
// of the first-pass encoding, r = |q - q_enc| of the query, P the relative
// error of the products and their FP32 accumulation, u = 2^-24.
// ---------------------------------------------------------------------------
struct CertArgs {
    float A;           // max ||x|| of the re-rank copy
    float Rx;          // max ||x - x_enc|| of the first pass's row encoding (0: exact)
    float P;           // relative product + accumulation error factor of the first pass
    int32_t d;
    const float *rq;   // [B] ||q - q_enc|| per query (NULL: the query is used exactly)
    const float *A2_dev;  // device max ||x||^2 (used instead of A when set)
};

__host__ __device__ inline float cert_bound(float qn, float rq, const CertArgs &c, int metric) {
    const float u = 5.9604645e-08f;   // 2^-24
    const float X = c.A + c.Rx;
    const float dot = qn * c.Rx + rq * X + c.P * (qn + rq) * X;
    const float e = metric == 0 ? 2.0f * dot + (float)(c.d + 32) * u * (qn * qn + c.A * c.A)
                                : dot + (float)(c.d + 32) * u * qn * c.A;
    return e * 1.0000153f + 1e-30f;   // (1 + 2^-16): the rounding of this formula
}

// Upper bound of the real-number k-th key given its FP32 direct-form value D.
__host__ __device__ inline float cert_rerank_up(float D, float qn, const CertArgs &c, int metric) {
    const float r = (float)(c.d + 8) * 1.1920929e-07f;   // (d + 8) 2^-23
    return metric == 0 ? D * (1.0f + r) + 1e-30f : D + r * qn * c.A + 1e-30f;
}

// Product error factors P of the first-pass kernels (see CertArgs).
__host__ __device__ inline float cert_P_ffma(int d) { return (float)(d + 16) * 1.1920929e-07f; }
__host__ __device__ inline float cert_P_tf32x3(int d) {
    return 4.0f * 9.5367432e-07f + (float)(3 * d + 16) * 1.1920929e-07f;   // 4 2^-20 + (3d+16) 2^-23
}
__host__ __device__ inline float cert_P_bf16x3(int d) {
    return 4.0f * 1.5258789e-05f + (float)(3 * d + 16) * 1.1920929e-07f;   // 4 2^-16 + (3d+16) 2^-23
}
__host__ __device__ inline float cert_P_bf16(int d) { return (float)(d + 16) * 1.1920929e-07f; }
__host__ __device__ inline float cert_P_e4m3(int d) { return (float)(d + 24) * 1.1920929e-07f; }

// Launch as a programmatic dependent of the previous kernel on the stream:
// the kernel may start while that kernel finishes, and must execute
// griddepcontrol.wait before reading anything it produced.
template <class... KArgs, class... Args>
inline cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                    cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

// ---------------------------------------------------------------------------
// Kernel launchers (each returns the launch error, if any).
// ---------------------------------------------------------------------------

// k_load.cu: load-time encodings and norms
cudaError_t launch_copy_f32(const float *src, int64_t n, int32_t d, float *dst, int32_t ld,
                            cudaStream_t s);
cudaError_t launch_bf16_to_f32(const uint16_t *src, int64_t n, int32_t d, float *dst,
                               int32_t ld, cudaStream_t s);
cudaError_t launch_copy_bf16(const uint16_t *src, int64_t n, int32_t d, uint16_t *dst,
                             int32_t ld, cudaStream_t s);
cudaError_t launch_f32_to_bf16(const float *src, int64_t n, int32_t d, int32_t lds,
                               uint16_t *dst, int32_t ld, cudaStream_t s);
cudaError_t launch_f32_to_e4m3(const float *src, int64_t n, int32_t d, int32_t lds,
                               uint8_t *dst, int32_t ld, float *scale, cudaStream_t s);
// bf16 pair copy of float32 rows (k_umma_pair.cu): dst [n x 2 ldp] uint16,
// row = [bf16(x) | bf16(x - bf16(x))], ldp = pair_ld(d) (a multiple of 64)
cudaError_t launch_f32_to_pair(const float *src, int64_t n, int32_t d, int32_t lds,
                               uint16_t *dst, int32_t ldp, cudaStream_t s);
cudaError_t launch_norms_f32(const float *x, int64_t n, int32_t d, int32_t ld, float *out,
                             cudaStream_t s);
cudaError_t launch_norms_bf16(const uint16_t *x, int64_t n, int32_t d, int32_t ld, float *out,
                              cudaStream_t s);

// Query preparation (a query batch on the device): float32 rows padded to
// the table's stride, and the per-query search state reset (global bound =
// kEmpty, candidate count = 0).
// dst [m x d] = rows ids[0..m) of src [* x d] (float32)
cudaError_t launch_gather_rows_f32(const float *src, int32_t d, const int32_t *ids, int64_t m,
                                   float *dst, cudaStream_t s);
cudaError_t launch_prep_queries(const float *q, int32_t B, int32_t d, float *qpad, int32_t ld,
                                uint64_t *tau_g, int32_t *cand_cnt, cudaStream_t s);

// k_filter.cu: predicate -> bitmap + per-tile counts -> offsets -> ids
cudaError_t launch_predicate(const AttrArg &attrs, int64_t n, const PredArg &p,
                             uint32_t *bitmap, int32_t *tile_counts, cudaStream_t s);
cudaError_t launch_tile_scan(const int32_t *tile_counts, int64_t n_tiles, int64_t *tile_offsets,
                             int64_t *total, cudaStream_t s);
cudaError_t launch_compact(const uint32_t *bitmap, int64_t n, const int64_t *tile_offsets,
                           int32_t *ids, cudaStream_t s);
// predicate -> unordered id list + count (one kernel; *count zero on entry)
// (pdev, when set, is a device copy of the predicate read instead of p)
cudaError_t launch_predicate_ids(const AttrArg &attrs, int64_t n, const PredArg &p,
                                 const PredArg *pdev, int32_t *ids, int64_t *count, int n_sm,
                                 cudaStream_t s);
// the selected rows among M evenly spaced rows (floor(i n / M), i < M), in any
// order; *count zero on entry, ids holds M entries
cudaError_t launch_sample_ids(const AttrArg &attrs, int64_t n, const PredArg &p, int64_t M,
                              int32_t *ids, int64_t *count, cudaStream_t s);

// k_scan_simt.cu: FP32 CUDA-core distance pass with per-CTA top-k'
struct ScanArgs {
    const void *X;         // [n x ld] rows: float32, or bf16 when x_bf16
    int32_t x_bf16;
    int32_t ld;            // row stride (elements), multiple of 16
    int32_t d;             // dimension (<= ld; columns d..ld-1 are zero)
    const float *xnorm;    // [n] ||x||^2
    const int32_t *ids;    // selected ids (NULL: dense scan of rows 0..n_rows-1)
    const uint32_t *bitmap;// dense scan only: predicate bitmap (NULL = all rows)
    const int64_t *count_dev; // device count of ids (ids mode) or NULL
    int64_t n_rows;        // rows (dense) or capacity bound (ids)
    const float *Q;        // [B x ld] float32 queries
    int32_t B;
    int32_t metric;        // 0 = L2, 1 = IP
    int32_t kp;            // candidates kept per (query, CTA)
    uint64_t *tau_g;       // [B] best known k'-th composite over all CTAs (kEmpty at start)
    int32_t *out_cnt;      // [B] appended candidates per query (0 at start)
    uint64_t *out;         // [B x out_cap] appended candidates
    int64_t out_cap;       // capacity per query (>= G * kp)
    float *keys_out;       // if set: write every first-pass key to keys_out[q * keys_ld + pos]
    int64_t keys_ld;       //   (+inf for padding) instead of selecting candidates,
    uint32_t *chunk_min;   //   and the smallest order-preserving key of each query over
    int64_t cmin_ld;       //   positions [128 c, 128 c + 128) to chunk_min[q * cmin_ld + c]
    int32_t *err;          // staged kernel: set to nonzero when a bounded wait gave up
    int32_t wait_test;     // tensor-core GEMV pass: 1 = first wait on a barrier nothing
                           // arrives at (the failure path of a bounded wait, for tests)
    int64_t *count_copy;   // dense-key forms (ids mode): block 0 stores *count_dev here
                           // for the merge, which may then clear *count_dev at once
};
cudaError_t launch_scan_simt(const ScanArgs &a, int grid_ctas, cudaStream_t s);
// Dense-key mode over an id list with rows staged by bulk asynchronous
// copies (one CTA per SM and query group); fits when a few stages of 128
// rows fit shared memory.
bool scan_keys_staged_fits(int B, int ld, int x_bf16);
cudaError_t launch_scan_keys_staged(const ScanArgs &a, int grid_ctas, cudaStream_t s);

// k_umma_rows.cu: the same dense-key distance pass for float32 rows on the
// tensor cores (rows as MMA M, queries as N, 3xTF32 split); grid_ctas row
// partitions per query tile of up to 64 queries.
bool umma_rows_fits(int B, int ld);
int umma_rows_grid(int B, int n_sm);
cudaError_t launch_umma_rows(const ScanArgs &a, int grid_ctas, cudaStream_t s);

int scan_simt_query_block(int B);

// k_umma_pair.cu: the same dense-key distance pass reading the bf16 pair
// copy (rows as MMA M, queries as N, 3 bf16 products); up to 64 queries.
int pair_ld(int d);
bool umma_pair_fits(int B, int d);
int umma_pair_grid(int B, int n_sm);
cudaError_t launch_umma_pair(const ScanArgs &a, const void *Xp, int grid_ctas, cudaStream_t s);

// k_probe.cu: measurement only -- read every listed row of a row-major
// [n_rows x row_bytes] table in full and add what was read into *out (ids
// outside [0, n_rows) are skipped).
cudaError_t launch_gather_probe(const void *rows, int64_t n_rows, int64_t row_bytes,
                                const int32_t *ids, int64_t m, float *out, int n_sm, cudaStream_t s);

// k_cells.cu: the batched plan over a table clustered by a two-column grid
// (per-query ranges on those columns).  Cells are (bin of column 0, bin of
// column 1), at most kGridMaxBins bins per column.
constexpr int kGridMaxBins = 64;
struct CellItem {      // work item: queries entries[q0 .. q0 + nq) of one cell
    int32_t cell, q0, nq, pad;
};
struct CellEntry {     // (query, cell) pair
    int32_t q;         // query; bit 31 set: the cell is not fully covered (test rows)
    int32_t chunk0;    // first 128-position chunk of the pair's key slot
};
struct CellArgs {
    CUtensorMap tmX;              // clustered bf16 rows (row_bytes), box 128 B x 128 rows
    const unsigned char *Q;       // [>= B x q_bytes] bf16 queries
    int32_t row_bytes;            // clustered row stride (>= 128, multiple of 16)
    int32_t q_bytes;              // query row stride (bytes past it read as zero)
    int32_t metric;
    const float *qnorm;           // [B] ||q||^2
    const float *xnorm;           // clustered ||x||^2
    const int32_t *a0, *a1;       // clustered grid columns
    const int32_t *qrange;        // [B x 4] inclusive ranges on column 0 and column 1
    const int64_t *cell_off;      // [cells + 1] first clustered row of each cell
    const CellItem *items;        // the work queue, largest items first
    int32_t n_items;
    int32_t *item_next;           // zeroed counter: the next item to take
    const CellEntry *entries;
    float *keys;                  // [chunks x 128] first-pass keys (+inf: not selected)
    uint32_t *chunk_min;          // [chunks] minimum of each chunk (order-preserving)
    int32_t *chunk_row;           // [chunks] clustered row of each chunk's first position
    int32_t *err;
};
bool cells_fit(int row_bytes);
cudaError_t launch_grid_cells(const int32_t *a0, const int32_t *a1, int64_t n, const int32_t *e0,
                              int nb0, const int32_t *e1, int nb1, int32_t *cell, int32_t *counts,
                              cudaStream_t s);
cudaError_t launch_grid_scatter(const int32_t *cell, int64_t n, const int64_t *off, int32_t *cursor,
                                int32_t *perm, cudaStream_t s);
// Clustered copies; rows of xg have gld >= ld elements (zero past ld).
cudaError_t launch_grid_gather(const int32_t *perm, int64_t n, const uint16_t *xb, int32_t ld,
                               int32_t gld, const float *norms, const int32_t *a0,
                               const int32_t *a1, uint16_t *xg, float *ng, int32_t *g0, int32_t *g1,
                               cudaStream_t s);
// cursor: 2 x cells zeroed counters
cudaError_t launch_cell_fill(const int32_t *rect, int32_t B, const int64_t *qchunk0,
                             const int32_t *nchunks, int nb1, int ncell, const int32_t *entry0,
                             int32_t *cursor, CellEntry *entries, cudaStream_t s);
// stages: 8, 6, 4, 3 or 2 row stages (0: the most that fit)
cudaError_t launch_cells_gemm(const CellArgs &a, int grid, int stages, cudaStream_t s);

// k_umma.cu: batched tensor-core distance pass (tcgen05) with per-query
// top-k' heaps in the epilogue
struct UmmaArgs {
    // TMA descriptors (byte-typed 2-D maps, 128-byte swizzle, box 128 bytes x
    // 256 rows for X and x 128 rows for Q); used when use_tma_* is set
    CUtensorMap tmX;
    CUtensorMap tmQ;
    int32_t use_tma_x;       // dense scans: row tiles by TMA
    int32_t use_tma_q;       // query tiles by TMA
    const unsigned char *X;  // encoded rows [n x row_bytes] (bf16 or E4M3)
    int32_t row_bytes;       // bytes per stored row (multiple of 16)
    const float *xnorm;      // [n] ||x||^2
    const float *xscale;     // [n] E4M3 row scales, or NULL
    const int32_t *ids;      // compacted ids, or NULL for a dense scan
    const uint32_t *bitmap;  // dense scan: predicate bitmap applied to scores (NULL = all)
    const int64_t *count_dev;
    int64_t n_rows;
    const unsigned char *Q;  // encoded queries [ceil(B/128)*128 x row_bytes], zero padded
    const float *qnorm;      // [B] ||q||^2
    const float *qscale;     // [B] E4M3 query scales, or NULL
    int32_t B;
    int32_t metric;
    int32_t kp;
    uint64_t *tau_g;         // [B] global bound
    int32_t *out_cnt;        // [B]
    uint64_t *out;           // [B x out_cap]
    int64_t out_cap;
    uint64_t *heap_g;        // global candidate buffers when the heaps do not fit in smem
                             // (umma_global_buffer_bytes(grid, kp) bytes)
    int32_t *err;            // set to nonzero when a bounded wait gave up
    // per-query predicates (batched launch): each query b keeps rows with
    // qrange[(b*nqc + c)*2] <= attr_c[row] <= qrange[(b*nqc + c)*2 + 1] for
    // every c < nqc (inclusive bounds); nqc == 0 disables it
    int32_t nqc;
    // per-query candidate width: k'_b = min(kp, max(kq[b] f, kq[b] + 8, 8 f)), f = kp_factor
    // when kq is set (batched launch with per-query k), else kp for every query
    const int32_t *kq;
    int32_t kp_factor;
    const int32_t *qcol[4];
    const int32_t *qrange;
};
constexpr int kMaxQCols = 4;
bool umma_config(int row_bytes, int kp, int *ns, bool *resa, size_t *smem, bool *heap_in_smem);
size_t umma_global_buffer_bytes(int grid, int kp);
// Encode a byte-typed 2-D tensor map over [rows x inner_bytes] with the
// 128-byte swizzle and a 128-byte x box_rows box.  False if unavailable.
bool make_tmap_2d(CUtensorMap *m, const void *base, uint64_t inner_bytes, uint64_t rows,
                  uint32_t box_rows);
cudaError_t launch_umma(const UmmaArgs &a, int dtype, int grid, cudaStream_t s);

// Tensor-path query encoding: qpad [B x ld] float32 -> Qenc rows of
// row_bytes (bf16 RNE, or E4M3 with a per-query scale max|q|/448), rows
// past B zeroed up to Bpad; qnorm[B] = ||q||^2 from the float32 values.
// qres (optional) [B] = ||q - q_enc|| (the decoded encoding, scale applied),
// rounded up, for the exactness certificate.
cudaError_t launch_prep_tensor_queries(const float *qpad, int32_t B, int32_t Bpad, int32_t d,
                                       int32_t ld, int dtype, unsigned char *Qenc,
                                       int32_t row_bytes, float *qnorm, float *qscale,
                                       float *qres, cudaStream_t s);
// Load-time statistics for the certificate: out[0] = max_i ||x_i|| over the
// float32 rows x [n x ld] (d values each), out[1] = max_i ||x_i - dec(enc(x_i))||
// for the encoding `dtype` (1 = bf16 copy xb [n x ld]; 2 = E4M3 codes x8 [n x
// ld] with row scales s8), both rounded up (float64 sums).  out must hold 2
// floats and start at 0.
cudaError_t launch_encoding_stats(const float *x, int64_t n, int32_t d, int32_t ld, int dtype,
                                  const uint16_t *xb, const uint8_t *x8, const float *s8,
                                  float *out, cudaStream_t s);
// Seed of a widened certifying pass: tau_g[b] = composite (T_b, UINT32_MAX)
// with T_b = dup[b] + E_b (the bound above for this pass's encoding and
// query b, |q_b| = sqrt(qnorm[b])), so the pass keeps every row whose
// first-pass key is <= T_b; cnt[b] = 0.
cudaError_t launch_cert_seed(const float *dup, const float *qnorm, CertArgs c, int metric,
                             int32_t B, uint64_t *tau_g, int32_t *cnt, cudaStream_t s);

// k_gemv.cu: fused FP32 scan for small batches (predicate on the fly, TMA
// bulk row gather, packed FP32 FMAs, per-CTA top-k')
struct GemvArgs {
    const float *X;        // [n x ld] float32 rows
    int32_t ld, d;
    const float *xnorm;    // [n]
    AttrArg attrs;
    PredArg pred;
    int64_t n;
    const float *Q;        // [B x ldq] float32 queries (ldq >= d)
    int32_t ldq;
    int32_t B, metric, kp;
    uint64_t *tau_g;       // [B] global bound (kEmpty at start)
    int32_t *out_cnt;      // [B] (0 at start)
    uint64_t *out;         // [B x out_cap]
    int64_t out_cap;
    int64_t *count_out;    // selected-row count accumulates here (may be NULL)
    int32_t *err;
};
size_t gemv_fused_smem(int QB, int ld, int kp);
int gemv_fused_query_block(int B);
cudaError_t launch_gemv_fused(const GemvArgs &a, int G, cudaStream_t s);

// k_merge.cu: merge the per-CTA candidates, exact FP32 re-rank, final top-k
// k_union.cu: the k best of the union of n_lists top-k lists per query
// (list l of query b at ids / dist [l * list_stride + b * k ...]), each row once
struct UnionArgs {
    const int64_t *ids;
    const float *dist;
    int64_t list_stride;   // entries between consecutive lists
    int32_t n_lists, k, B, metric;
    int64_t *out_ids;      // [B x k]
    float *out_dist;
};
int union_max_entries();   // largest n_lists x k
// Row-id offset added to the ids of list l < n (row-sharded tables: the
// global id of shard l's row 0), passed by value.
constexpr int kMaxLists = 64;
struct ListOffsets {
    int32_t n;
    int64_t v[kMaxLists];
};
cudaError_t launch_union_topk(const UnionArgs &a, cudaStream_t s, const ListOffsets *off = nullptr);

// k_range.cu: filtered range search on the dense key matrix
struct RangeArgs {
    float *keys;               // [B x keys_ld] first-pass keys; the mark pass leaves
                               // each result's exact score there and +inf elsewhere
    int64_t keys_ld;
    uint32_t *chunk_min;       // [B x cmin_ld] ordered chunk minima; afterwards 0 for
                               // a chunk with results, ~0 otherwise
    int64_t cmin_ld;
    const int32_t *ids;        // [count] row id of each position
    const int64_t *count_dev;  // selected rows
    const float *X;            // [n x ld] float32 rows
    int32_t ld, d;
    const float *Q;            // [B x ld] queries, zero past d
    const float *xn_max;       // max ||x||^2 over the rows (one float)
    int32_t B;
    int32_t metric;            // 0: squared L2 <= eps; 1: q.x >= eps
    float eps;
    int64_t *counts;           // [B] results per query (mark pass)
    const int64_t *offsets;    // [B + 1] result offsets (write pass)
    int64_t *out_ids;          // [offsets[B]]
    float *out_dist;           // [offsets[B]] squared distance or q.x
};
cudaError_t launch_max_f32(const float *v, int64_t n, float *out, cudaStream_t s);
cudaError_t launch_range_mark(const RangeArgs &a, cudaStream_t s);
cudaError_t launch_range_write(const RangeArgs &a, cudaStream_t s);

struct MergeArgs {
    const uint64_t *cand;  // [B x m] composites (per-query row stride m)
    int64_t m;
    const int32_t *cand_cnt; // [B] valid entries per query (NULL: all m, kEmpty = none)
    int32_t kp;            // candidates to re-rank per query
    const int32_t *k;      // [B] or NULL (k_shared)
    int32_t k_shared;
    int32_t k_max;
    int32_t B;
    int32_t metric;
    int32_t rerank;        // 1 = exact FP32 re-rank; 0 = keep first-pass keys
    const float *Xf;       // float32 master rows (or NULL)
    const uint16_t *Xb;    // bf16 master rows when no float32 copy
    int32_t ld;            // stride of the master copy
    int32_t d;
    const float *Q;        // [B x ldq] float32 queries
    int32_t ldq;
    int64_t *out_ids;      // [B x k_max]
    float *out_dist;       // [B x k_max]
    uint64_t *reset_tau;   // if set: tau[b] = kEmpty and cand_cnt[b] = 0 after the merge
    int64_t *reset_count;  // if set: *reset_count = 0 after the merge (block 0)
    int32_t stage_cap;     // candidates per query staged in shared memory (0 = none)
    int32_t kp_factor;     // f > 0 and k set: query b re-ranks min(kp, max(k[b] f, k[b] + 8, 8 f))
    // Dense-key front end (launch_keys_merge): query b's candidates are
    // positions 0..*key_count-1 of row b of the first-pass key matrix.
    const float *keys;     // [B x keys_ld] (keys_ld a multiple of 4 for vector loads)
    int64_t keys_ld;
    const int32_t *key_ids;      // position -> row id (NULL: position is the row)
    const int64_t *key_count;    // positions per query (device)
    // Per-query rows (the cell plan; row_chunk0 NULL: the matrix above).
    // Query b's keys are chunks row_chunk0[b] .. row_chunk0[b+1] of keys and
    // chunk_min; position p of chunk c is clustered row chunk_row[c] + p % 128,
    // original row row_ids[that].
    const int64_t *row_chunk0;
    const int32_t *chunk_row;
    const int32_t *row_ids;
    const uint32_t *chunk_min;   // [B x cmin_ld] per-128-position minima (ordered keys)
    int64_t cmin_ld;
    int32_t *done;         // zero-initialised counter: the last CTA clears *reset_count
    // Exactness certificate (cert_flag NULL: none).  Per query b:
    //   cert_flag[b] = 0 certified, 1 not certified (cert_dup[b] = the k-th exact
    //   key rounded up, for a wider pass), 2 certified after the in-kernel
    //   fallback of the dense-key merge (every row whose first-pass key is
    //   within the bound re-ranked exactly).
    CertArgs cert;
    int32_t *cert_flag;
    float *cert_dup;
    // Optional summary word (merge_rerank): raised to 1 when a query is not
    // certified, to 2 when *scan_err (the distance pass's error word) is set.
    int32_t *status;
    const int32_t *scan_err;
    // merge_rerank: 1 = only report, per query, the k-th exact key rounded up
    // (+inf when fewer than k candidates) in cert_dup -- a pass over a sample
    // of the selected rows, whose k-th exact distance bounds the whole
    // selection's from above
    int32_t dup_only;
    // keys_merge_kernel: if set, block 0 copies *err_src to *err_dst at its
    // end (the distance pass's error word to a page-locked host word)
    const int32_t *err_src;
    int32_t *err_dst;
};
cudaError_t launch_merge_rerank(const MergeArgs &a, cudaStream_t s);
// tau_g[b] = (k'-th smallest of cand[b][0 .. min(cnt[b], m))) + 1, or kEmpty
// with fewer than k' entries; cnt[b] = 0 afterwards.  k' = kp, or with kq
// min(kp, max(kq[b] f, kq[b] + 8, 8 f)) for f = kp_factor.
cudaError_t launch_seed_bound(const uint64_t *cand, int64_t m, int32_t *cnt, int B, int kp,
                              const int32_t *kq, int kp_factor, uint64_t *tau_g, cudaStream_t s);
// Staged results of a query subset back into the outputs: row i of sid/sd
// ([m x k_max]) becomes row idx[i] of oid/od unless flag[i] == 1 (not
// certified); flag NULL copies every row.
cudaError_t launch_scatter_topk(const int64_t *sid, const float *sd, const int32_t *idx,
                                const int32_t *flag, int64_t m, int32_t k_max, int64_t *oid,
                                float *od, cudaStream_t s);
// cap: per-query survivor list capacity in shared memory; beyond it a query
// is selected from its whole key row.
size_t keys_merge_smem(int kp, int cap, int ld);
// dynamic shared memory the dense-key merge can have next to its static arrays
size_t keys_merge_max_smem();
cudaError_t launch_keys_merge(const MergeArgs &a, int cap, cudaStream_t s);

}  // namespace vrs
