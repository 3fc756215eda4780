// k_cells.cu -- the batched plan over a table clustered by a two-column
// grid: many queries, each with its own conjunction of ranges on two
// attribute columns (the batched "N:N" Tensor formulation of Sec. 3.1 with
// the predicate of Sec. 3.2 applied per query).
//
// Grid (vrs_build_grid): the values of two attribute columns are cut at
// sample quantiles into nb0 x nb1 bins; every row falls into one cell (its
// bin of each column), and a clustered copy of the table -- bf16 rows,
// norms, the two columns, the original row id -- stores the rows cell by
// cell.  A query selects rows only from the cells its two ranges overlap,
// and in the cells both ranges cover entirely every row qualifies, so only
// the boundary cells test rows one by one.
//
// Per batch each (query, overlapped cell) pair owns a key slot of
// ceil(n_cell / 128) chunks of 128 positions.  A query's slots are
// contiguous: they form its row of the dense first-pass key matrix, which
// keys_merge_kernel reads as in the GEMV plan (chunk minima, bound,
// candidate chunks, exact re-rank, certificate).  Work items are (cell, up
// to 128 of the cell's queries).  cells_gemm_kernel runs one CTA per SM; the
// CTAs take items from a work queue (an atomic counter over the items,
// largest first), the query loader taking each next item for its CTA.  A
// tile is one 128-row chunk of the cell (MMA M, TMEM lanes) against the
// item's queries (MMA N = their count rounded up to 16), so a warp's key
// stores for one query are 128 contiguous bytes:
//   warp 0     TMA loads of the cell's rows, 128 rows x 128 bytes per stage;
//   warp 1     the item's queries, gathered with cp.async (double-buffered
//              across items);
//   warp 2     TMEM allocation and tcgen05.mma (bf16, fp32 accumulators:
//              two tiles, so the epilogue of one overlaps the MMAs of the
//              next);
//   warps 3-18 epilogue: warp (lane quarter, part) takes 32 rows and a
//              quarter of the item's queries; per row and query the key
//              ||q||^2 - 2 q.x + ||x||^2 (L2) or -q.x (IP), +inf where a
//              boundary cell's row fails the query's ranges or past the
//              cell's end; the keys, each query's chunk minimum (over the
//              four lane quarters) and the chunk's first clustered row are
//              written.
// Every mbarrier wait is bounded; on timeout the kernel raises *err, lets
// copies and MMAs drain, frees its TMEM and returns.
#include <cudaTypedefs.h>

#include <algorithm>

#include "umma.cuh"
#include "vrs_internal.cuh"

namespace vrs {
namespace {

using namespace umma;

constexpr int kCM = 128;               // rows per tile (MMA M, TMEM lanes): one key chunk
constexpr int kCQ = 128;               // queries per item (MMA N at most)
constexpr int kCK = 128;               // bytes of K per block
constexpr int kCEpi = 512;              // 16 epilogue warps: four per TMEM lane quarter
constexpr int kCThreads = 96 + kCEpi;
constexpr uint32_t kCCols = 256;        // two accumulators of up to 128 columns
constexpr int kQBlock = kCQ * kCK;     // 16 KB: one K block of the query tile
constexpr int kRStage = kCM * kCK;     // 16 KB: one K block of a row tile

struct CLayout {
    int nkb, ns;
    size_t q_off, r_off, qi_off, cm_off, bar_off, total;
};

// Per-query values of the current item in shared memory (slot j).
struct QInfo {
    float qn;         // ||q||^2 (L2)
    int32_t partial;  // 1: test the rows against the ranges
    float *slot;      // the (query, cell) key slot's first position (NULL: no query)
};

__host__ __device__ inline CLayout cell_layout(int row_bytes, int ns) {
    CLayout L;
    L.nkb = (row_bytes + kCK - 1) / kCK;
    L.ns = ns;
    size_t off = 0;
    L.q_off = off;
    off += (size_t)2 * L.nkb * kQBlock;   // query tiles of two items
    L.r_off = off;
    off += (size_t)ns * kRStage;          // row stages
    L.qi_off = off;
    off += (size_t)2 * kCQ * (sizeof(QInfo) + 16);   // two items' QInfo and ranges
    L.cm_off = off;
    off += (size_t)2 * 4 * kCQ * 4;       // chunk minima per lane quarter, two tiles
    L.bar_off = off;
    off += (2 * ns + 8 + 1) * 8 + 16;     // full, empty, accfull x2, accempty x2, qfull x2, qempty x2, done; tmem, abort, item x2
    L.total = off + 1024;                 // slack for 1024-byte alignment
    return L;
}

// Barrier of the epilogue threads with an OR of a flag, so that every
// epilogue warp takes the same decision.
__device__ __forceinline__ bool epi_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, 512, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

// Bins of a value: the number of inner boundaries e[0..m) at or below v.
__device__ __forceinline__ int bin_of(const int32_t *e, int m, int32_t v) {
    int lo = 0, hi = m;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (e[mid] <= v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- grid build

__global__ void __launch_bounds__(256)
grid_cell_kernel(const int32_t *__restrict__ a0, const int32_t *__restrict__ a1, int64_t n,
                 const int32_t *__restrict__ e0, int nb0, const int32_t *__restrict__ e1, int nb1,
                 int32_t *__restrict__ cell, int32_t *__restrict__ counts) {
    __shared__ int32_t s0[kGridMaxBins], s1[kGridMaxBins];
    __shared__ int32_t hist[kGridMaxBins * kGridMaxBins];
    const int nc = nb0 * nb1;
    for (int i = threadIdx.x; i < nb0 - 1; i += blockDim.x) s0[i] = e0[i];
    for (int i = threadIdx.x; i < nb1 - 1; i += blockDim.x) s1[i] = e1[i];
    for (int i = threadIdx.x; i < nc; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int c = bin_of(s0, nb0 - 1, a0[r]) * nb1 + bin_of(s1, nb1 - 1, a1[r]);
        cell[r] = c;
        atomicAdd(&hist[c], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nc; i += blockDim.x)
        if (hist[i]) atomicAdd(&counts[i], hist[i]);
}

// Clustered position of every row: the cell's first row plus an arrival
// rank (lanes of a warp that share a cell take one atomic).
__global__ void __launch_bounds__(256)
grid_scatter_kernel(const int32_t *__restrict__ cell, int64_t n, const int64_t *__restrict__ off,
                    int32_t *__restrict__ cursor, int32_t *__restrict__ perm) {
    const int lane = threadIdx.x & 31;
    for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x; r0 < n; r0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = r0 + threadIdx.x;
        const int c = r < n ? cell[r] : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, c);
        const int leader = __ffs(grp) - 1;
        const int rank = __popc(grp & ((1u << lane) - 1));
        int base = 0;
        if (c >= 0 && lane == leader) base = atomicAdd(&cursor[c], __popc(grp));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (c >= 0) perm[off[c] + base + rank] = (int32_t)r;
    }
}

// Clustered copies: row pos of the copy is row perm[pos] of the table.
__global__ void __launch_bounds__(256)
grid_gather_kernel(const int32_t *__restrict__ perm, int64_t n, const uint16_t *__restrict__ xb,
                   int32_t ld, int32_t gld, const float *__restrict__ norms,
                   const int32_t *__restrict__ a0, const int32_t *__restrict__ a1,
                   uint16_t *__restrict__ xg, float *__restrict__ ng, int32_t *__restrict__ g0,
                   int32_t *__restrict__ g1) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t ws = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int n16 = ld / 8, g16 = gld / 8;   // 16-byte pieces of a row
    for (int64_t p = w0; p < n; p += ws) {
        const int64_t r = perm[p];
        const uint4 *src = reinterpret_cast<const uint4 *>(xb + r * ld);
        uint4 *dst = reinterpret_cast<uint4 *>(xg + p * gld);
        for (int i = lane; i < g16; i += 32) dst[i] = i < n16 ? src[i] : make_uint4(0, 0, 0, 0);
        if (lane == 0) {
            ng[p] = norms[r];
            g0[p] = a0[r];
            g1[p] = a1[r];
        }
    }
}

// ---------------------------------------------------------------- per batch

// One warp per query: the (query, cell) pairs of its rectangle of cells, in
// row-major cell order, each with its key slot (consecutive chunks from the
// query's first chunk), put in the cell's list: fully covered pairs from
// the front (cursor[c]), the others from the back (cursor[cells + c]).
// rect[q] = bin ranges (b0lo, b0hi, b1lo, b1hi) and the fully covered bins
// (f0lo, f0hi, f1lo, f1hi); empty cells get no pair.
__global__ void __launch_bounds__(256)
cell_fill_kernel(const int32_t *__restrict__ rect, int32_t B, const int64_t *__restrict__ qchunk0,
                 const int32_t *__restrict__ nchunks, int nb1, int ncell,
                 const int32_t *__restrict__ entry0, int32_t *__restrict__ cursor,
                 CellEntry *__restrict__ entries) {
    const int lane = threadIdx.x & 31;
    const int q = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (q >= B) return;
    const int32_t *rq = rect + (int64_t)q * 8;
    const int b0lo = rq[0], b0hi = rq[1], b1lo = rq[2], b1hi = rq[3];
    const int f0lo = rq[4], f0hi = rq[5], f1lo = rq[6], f1hi = rq[7];
    int64_t base = qchunk0[q];
    for (int b0 = b0lo; b0 <= b0hi; ++b0) {
        for (int j = b1lo; j <= b1hi; j += 32) {
            const int b1 = j + lane;
            const int c = b0 * nb1 + b1;
            const int nch = b1 <= b1hi ? nchunks[c] : 0;
            int incl = nch;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (nch > 0) {
                const bool full = b0 >= f0lo && b0 <= f0hi && b1 >= f1lo && b1 <= f1hi;
                const int slot = full ? entry0[c] + atomicAdd(&cursor[c], 1)
                                      : entry0[c + 1] - 1 - atomicAdd(&cursor[ncell + c], 1);
                CellEntry en;
                en.q = full ? q : (int32_t)((uint32_t)q | 0x80000000u);
                en.chunk0 = (int32_t)(base + incl - nch);
                entries[slot] = en;
            }
            base += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

// ---------------------------------------------------------------- the GEMM

// Ties 32 registers written by an asynchronous tcgen05.ld to this point
// (after tcgen05.wait::ld), so no use of them is scheduled before it.
__device__ __forceinline__ void reg_fence32(uint32_t (&r)[32]) {
#pragma unroll
    for (int i = 0; i < 32; i += 8)
        asm volatile("" : "+r"(r[i]), "+r"(r[i + 1]), "+r"(r[i + 2]), "+r"(r[i + 3]), "+r"(r[i + 4]),
                     "+r"(r[i + 5]), "+r"(r[i + 6]), "+r"(r[i + 7]));
}

__device__ __forceinline__ bool cwarp_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
    const bool ok = mbar_wait(bar, parity, abort);
    return __all_sync(0xffffffffu, ok);
}

// MET: 0 = L2, 1 = inner product.
template <int NS, int MET>
__global__ void __launch_bounds__(kCThreads, 1)
cells_gemm_kernel(const __grid_constant__ CellArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw_u32 = smem_u32(smem_raw);
    unsigned char *sm = smem_raw + (((raw_u32 + 1023u) & ~1023u) - raw_u32);
    const CLayout L = cell_layout(a.row_bytes, NS);
    const int nkb = L.nkb;
    unsigned char *Qsm = sm + L.q_off;
    unsigned char *Rsm = sm + L.r_off;
    QInfo *qinfo = reinterpret_cast<QInfo *>(sm + L.qi_off);                 // [2][kCQ]
    int4 *qrng = reinterpret_cast<int4 *>(qinfo + 2 * kCQ);                   // [2][kCQ]
    uint32_t *cmin_s = reinterpret_cast<uint32_t *>(sm + L.cm_off);          // [2][4][kCQ]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L.bar_off);
    uint64_t *full = bars, *empty = bars + NS, *accfull = bars + 2 * NS,
             *accempty = bars + 2 * NS + 2, *qfull = bars + 2 * NS + 4, *qempty = bars + 2 * NS + 6,
             *done = bars + 2 * NS + 8;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * NS + 9);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    // the item of each query buffer, taken from the work queue by the loader
    // (-1: the queue is empty); published with the buffer's qfull phase
    volatile int32_t *item_slot = reinterpret_cast<volatile int32_t *>(tmem_slot + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accfull[i], 1);
            mbar_init(&accempty[i], kCEpi / 32);
            mbar_init(&qfull[i], 32);
            // the item's MMAs (one commit) and its epilogue (every warp)
            mbar_init(&qempty[i], 1 + kCEpi / 32);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 2) {
        tmem_alloc(tmem_slot, kCCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    auto fail = [&]() {
        *abort_flag = 1;
        atomicExch(a.err, 1);
    };
    auto tiles_of = [&](const CellItem &w, int64_t *r0, int64_t *r1) {
        *r0 = a.cell_off[w.cell];
        *r1 = a.cell_off[w.cell + 1];
        return (int)((*r1 - *r0 + kCM - 1) / kCM);
    };

    if (warp == 0) {
        // ------------------------------------------------ row tiles by TMA
        int it = 0;
        bool ok = true;
        for (int u = 0; ok; ++u) {
            const int ab = u & 1;
            if (!cwarp_wait(&qfull[ab], (u >> 1) & 1, abort_flag)) {
                if (lane == 0) fail();
                ok = false;
                break;
            }
            const int i = item_slot[ab];
            if (i < 0) break;
            const CellItem w = a.items[i];
            int64_t r0, r1;
            const int T = tiles_of(w, &r0, &r1);
            for (int t = 0; t < T && ok; ++t)
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int st = it % NS;
                    if (!cwarp_wait(&empty[st], ((it / NS) & 1) ^ 1, abort_flag)) {
                        if (lane == 0) fail();
                        ok = false;
                        break;
                    }
                    if (lane == 0) {
                        // the stage completes on the box's bytes and this arrival
                        mbar_expect_tx(&full[st], (uint32_t)kRStage);
                        tma_load_2d(smem_u32(Rsm + (size_t)st * kRStage), &a.tmX, kb * kCK,
                                    (int32_t)(r0 + (int64_t)t * kCM), &full[st]);
                        mbar_arrive(&full[st]);
                    }
                    __syncwarp();
                }
        }
        // copies still in flight land before the CTA leaves (bounded wait)
        if (!ok && lane == 0) {
            volatile int never = 0;
            for (int j = it > NS ? it - NS : 0; j < it; ++j) mbar_wait(&full[j % NS], (j / NS) & 1, &never);
        }
    } else if (warp == 1) {
        // ------------------------------------------------ query tiles and values
        for (int u = 0;; ++u) {
            const int ab = u & 1;
            if (!cwarp_wait(&qempty[ab], ((u >> 1) & 1) ^ 1, abort_flag)) {
                if (lane == 0) fail();
                break;
            }
            // the next item of the work queue (largest first)
            int i = 0;
            if (lane == 0) i = atomicAdd(a.item_next, 1);
            i = __shfl_sync(0xffffffffu, i, 0);
            if (i >= a.n_items) {
                if (lane == 0) item_slot[ab] = -1;
                mbar_arrive(&qfull[ab]);
                break;
            }
            if (lane == 0) item_slot[ab] = i;
            const CellItem w = a.items[i];
            unsigned char *qt = Qsm + (size_t)ab * nkb * kQBlock;
            for (int r = lane; r < kCQ; r += 32) {
                CellEntry en{0, -1};
                if (r < w.nq) en = a.entries[w.q0 + r];
                const int32_t q = r < w.nq ? (en.q & 0x7fffffff) : -1;
                const unsigned char *qrow = a.Q + (int64_t)(q < 0 ? 0 : q) * a.q_bytes;
                for (int kb = 0; kb < nkb; ++kb)
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const int off = kb * kCK + c * 16;
                        const uint32_t nb = (q >= 0 && off < a.q_bytes) ? 16u : 0u;
                        cp_async16(smem_u32(qt + (size_t)kb * kQBlock + sw128_offset(r, c)),
                                   nb ? qrow + off : a.Q, nb);
                    }
                QInfo qi{0.0f, 0, nullptr};
                int4 rg = make_int4(INT32_MIN, INT32_MAX, INT32_MIN, INT32_MAX);
                if (q >= 0) {
                    qi.qn = a.metric == 0 ? a.qnorm[q] : 0.0f;
                    qi.slot = a.keys + (int64_t)en.chunk0 * kCM;
                    qi.partial = en.q < 0 ? 1 : 0;
                    if (qi.partial) rg = *reinterpret_cast<const int4 *>(a.qrange + (int64_t)q * 4);
                }
                qinfo[ab * kCQ + r] = qi;
                qrng[ab * kCQ + r] = rg;
            }
            cp_async_commit();
            cp_async_wait<0>();
            fence_proxy_async_smem();
            mbar_arrive(&qfull[ab]);   // (releases the QInfo stores too)
        }
    } else if (warp == 2) {
        // ------------------------------------------------ MMA issue
        if (lane == 0) {
            int it = 0, tc = 0;
            bool ok = true;
            for (int u = 0; ok; ++u) {
                const int ab = u & 1;
                if (!mbar_wait(&qfull[ab], (u >> 1) & 1, abort_flag)) {
                    fail();
                    break;
                }
                tc_fence_after();
                const int i = item_slot[ab];
                if (i < 0) break;
                const CellItem w = a.items[i];
                int64_t r0, r1;
                const int T = tiles_of(w, &r0, &r1);
                const uint32_t nq16 = (uint32_t)((w.nq + 15) & ~15);
                const uint32_t id = idesc(1, kCM, nq16);
                const uint32_t qbase = smem_u32(Qsm + (size_t)ab * nkb * kQBlock);
                for (int t = 0; t < T && ok; ++t, ++tc) {
                    const int acc = tc & 1, use = tc >> 1;
                    if (!mbar_wait(&accempty[acc], (use & 1) ^ 1, abort_flag)) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem_base + (uint32_t)(acc * kCQ);
                    for (int kb = 0; kb < nkb; ++kb, ++it) {
                        const int st = it % NS;
                        if (!mbar_wait(&full[st], (it / NS) & 1, abort_flag)) {
                            fail();
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t rb = smem_u32(Rsm + (size_t)st * kRStage);
                        const uint32_t qb = qbase + (uint32_t)(kb * kQBlock);
#pragma unroll
                        for (int kk = 0; kk < kCK / 32; ++kk)
                            mma_f16(d, desc_sw128(rb + kk * 32), desc_sw128(qb + kk * 32), id,
                                    (kb | kk) != 0 ? 1u : 0u);
                        mma_commit(&empty[st]);
                    }
                    if (!ok) break;
                    mma_commit(&accfull[acc]);
                }
                mma_commit(&qempty[ab]);
            }
            mma_commit(done);
            if (!mbar_wait(done, 0, abort_flag)) {
                volatile int never = 0;
                mbar_wait(done, 0, &never);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue
        const int et = tid - 96;                 // 0..511
        const int ew = warp - 3;                 // 0..15
        const int lq = warp & 3;                 // TMEM lane quarter of this warp
        const int qq = ew >> 2;                  // its part of the item's queries
        const int row = lq * 32 + lane;          // row within the tile
        const float kInf = __int_as_float(0x7f800000);
        int tc = 0;
        bool ok = true;
        for (int u = 0; ok; ++u) {
            const int ab = u & 1;
            // the item and its query values (the loader refills this buffer
            // only after every epilogue warp released it, below)
            if (!cwarp_wait(&qfull[ab], (u >> 1) & 1, abort_flag)) {
                if (lane == 0) fail();
                ok = false;
            }
            if (epi_or(!ok)) {
                ok = false;
                break;
            }
            const int i = item_slot[ab];
            if (i < 0) break;
            const CellItem w = a.items[i];
            int64_t r0, r1;
            const int T = tiles_of(w, &r0, &r1);
            const int64_t nrow = r1 - r0;
            // queries [jq, jq + jn) of the item: four balanced parts of at most 32
            const int per = (w.nq + 3) >> 2;
            const int jq = qq * per;
            const int jn = max(0, min(per, w.nq - jq));
            const QInfo *qi = qinfo + ab * kCQ;
            const int4 *qr = qrng + ab * kCQ;
            float xn = 0.0f;
            int32_t x0 = 0, x1 = 0;
            auto fetch = [&](int t) {
                const int64_t p = r0 + (int64_t)t * kCM + row;
                const bool in = p < r1;
                xn = (in && MET == 0) ? a.xnorm[p] : 0.0f;
                x0 = in ? a.a0[p] : 0;
                x1 = in ? a.a1[p] : 0;
            };
            fetch(0);
            for (int t = 0; t < T; ++t, ++tc) {
                const int acc = tc & 1, use = tc >> 1;
                const float xr = xn;
                const int32_t y0 = x0, y1 = x1;
                const int pos = t * kCM + row;   // position in the (query, cell) key slot
                const bool in = pos < nrow;
                const bool full_tile = (int64_t)(t + 1) * kCM <= nrow;
                if (t + 1 < T) fetch(t + 1);
                if (!cwarp_wait(&accfull[acc], use & 1, abort_flag)) {
                    if (lane == 0) fail();
                    ok = false;
                }
                tc_fence_after();
                uint32_t *cm = cmin_s + (tc & 1) * 4 * kCQ + lq * kCQ;
                if (ok && jn > 0) {
                    uint32_t v[32];
                    tmem_ld32(tmem_base + ((uint32_t)(lq * 32) << 16) + (uint32_t)(acc * kCQ + jq), v);
                    tmem_ld_wait();
                    reg_fence32(v);
                    auto one = [&](int c) {
                        const int j = jq + c;
                        const QInfo qv = qi[j];
                        const float sv = __uint_as_float(v[c]);
                        float k;
                        uint32_t ko;
                        if (MET == 0) {
                            k = fmaxf(fmaf(-2.0f, sv, qv.qn + xr), 0.0f);
                        } else {
                            k = 0.0f - sv;   // (a zero key is +0, as the minima assume)
                        }
                        if (qv.partial) {
                            const int4 rg = qr[j];
                            if (!(y0 >= rg.x && y0 <= rg.y && y1 >= rg.z && y1 <= rg.w)) k = kInf;
                        }
                        if (!full_tile && !in) k = kInf;
                        // order-preserving bits; an L2 key is never negative
                        ko = MET == 0 ? (__float_as_uint(k) | 0x80000000u) : float_to_ordered(k);
                        qv.slot[pos] = k;
                        const uint32_t m = __reduce_min_sync(0xffffffffu, ko);
                        if (lane == 0) cm[j] = m;
                    };
                    if (jn == 32) {
#pragma unroll
                        for (int c = 0; c < 32; ++c) one(c);
                    } else {
#pragma unroll
                        for (int c = 0; c < 32; ++c)
                            if (c < jn) one(c);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&accempty[acc]);
                // the four lane quarters' minima of this tile -> each query's chunk minimum
                ok = !epi_or(!ok || *abort_flag);
                if (ok && et < w.nq) {
                    const uint32_t *c4 = cmin_s + (tc & 1) * 4 * kCQ;
                    const uint32_t m = min(min(c4[et], c4[kCQ + et]), min(c4[2 * kCQ + et], c4[3 * kCQ + et]));
                    const int64_t ch = (qi[et].slot - a.keys) / kCM + t;
                    a.chunk_min[ch] = m;
                    a.chunk_row[ch] = (int32_t)(r0 + (int64_t)t * kCM);
                }
                if (!ok) break;
            }
            if (lane == 0) mbar_arrive(&qempty[ab]);
            ok = !epi_or(!ok);   // every epilogue warp leaves the item together
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kCCols);
    }
}

constexpr size_t kCSmemMax = 227 * 1024;

int cells_stages(int row_bytes) {
    for (int ns : {8, 6, 4, 3, 2})
        if (cell_layout(row_bytes, ns).total <= kCSmemMax) return ns;
    return 0;
}

template <int NS>
cudaError_t launch_cells_t(const CellArgs &a, int grid, cudaStream_t s) {
    if (cell_layout(a.row_bytes, NS).total > kCSmemMax) return cudaErrorInvalidValue;
    const size_t smem = cell_layout(a.row_bytes, NS).total;
    auto k = a.metric == 0 ? cells_gemm_kernel<NS, 0> : cells_gemm_kernel<NS, 1>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kCThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool cells_fit(int row_bytes) {
    return row_bytes % 16 == 0 && row_bytes >= kCK && cells_stages(row_bytes) >= 2;
}

cudaError_t launch_grid_cells(const int32_t *a0, const int32_t *a1, int64_t n, const int32_t *e0,
                              int nb0, const int32_t *e1, int nb1, int32_t *cell, int32_t *counts,
                              cudaStream_t s) {
    if (!a0 || !a1 || !cell || !counts || n < 1 || nb0 < 1 || nb1 < 1 || nb0 > kGridMaxBins ||
        nb1 > kGridMaxBins)
        return cudaErrorInvalidValue;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    grid_cell_kernel<<<blocks, 256, 0, s>>>(a0, a1, n, e0, nb0, e1, nb1, cell, counts);
    return cudaGetLastError();
}

cudaError_t launch_grid_scatter(const int32_t *cell, int64_t n, const int64_t *off, int32_t *cursor,
                                int32_t *perm, cudaStream_t s) {
    if (!cell || !off || !cursor || !perm || n < 1) return cudaErrorInvalidValue;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8192);
    grid_scatter_kernel<<<blocks, 256, 0, s>>>(cell, n, off, cursor, perm);
    return cudaGetLastError();
}

cudaError_t launch_grid_gather(const int32_t *perm, int64_t n, const uint16_t *xb, int32_t ld,
                               int32_t gld, const float *norms, const int32_t *a0,
                               const int32_t *a1, uint16_t *xg, float *ng, int32_t *g0, int32_t *g1,
                               cudaStream_t s) {
    if (!perm || !xb || !norms || !a0 || !a1 || !xg || !ng || !g0 || !g1 || n < 1 || ld % 8 ||
        gld % 8 || gld < ld)
        return cudaErrorInvalidValue;
    const int blocks = (int)std::min<int64_t>((n * 32 + 255) / 256, 16384);
    grid_gather_kernel<<<blocks, 256, 0, s>>>(perm, n, xb, ld, gld, norms, a0, a1, xg, ng, g0, g1);
    return cudaGetLastError();
}

cudaError_t launch_cell_fill(const int32_t *rect, int32_t B, const int64_t *qchunk0,
                             const int32_t *nchunks, int nb1, int ncell, const int32_t *entry0,
                             int32_t *cursor, CellEntry *entries, cudaStream_t s) {
    if (!rect || !qchunk0 || !nchunks || !entry0 || !cursor || !entries || B < 1 || ncell < 1)
        return cudaErrorInvalidValue;
    cell_fill_kernel<<<(unsigned)(((int64_t)B * 32 + 255) / 256), 256, 0, s>>>(
        rect, B, qchunk0, nchunks, nb1, ncell, entry0, cursor, entries);
    return cudaGetLastError();
}

cudaError_t launch_cells_gemm(const CellArgs &a, int grid, int stages, cudaStream_t s) {
    if (!a.err || !a.items || !a.entries || !a.keys || !a.chunk_min || !a.chunk_row ||
        !a.item_next || grid < 1 || a.n_items < 1 || !cells_fit(a.row_bytes) || a.q_bytes % 16 ||
        a.q_bytes > a.row_bytes)
        return cudaErrorInvalidValue;
    switch (stages > 0 ? stages : cells_stages(a.row_bytes)) {
        case 8: return launch_cells_t<8>(a, grid, s);
        case 6: return launch_cells_t<6>(a, grid, s);
        case 4: return launch_cells_t<4>(a, grid, s);
        case 3: return launch_cells_t<3>(a, grid, s);
        case 2: return launch_cells_t<2>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace vrs
