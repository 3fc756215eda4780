// k_umma.cu -- the batched "Tensor formulation" of the scan (Sec. 3.1, N:N:
// a batch of queries against a batch of rows as one matrix product), on the
// 5th-generation tensor cores (tcgen05, accumulators in tensor memory).
//
// One CTA = one tile of 128 queries (MMA M) against a contiguous range of
// selected rows, consumed 256 rows (MMA N) at a time.  Rows are either the
// compacted ids of the qualifying rows (predicate first, late
// materialisation, Sec. 3.2 / Fig. 3 -- gathered straight into shared
// memory, never copied to a dense matrix), or every row with the predicate
// bitmap applied to the scores (the on-the-fly strategy of Sec. 3.2).
//
// Warp roles (416 threads):
//   warps 0-7  producers: cp.async 16-byte gathers of the row tiles (and the
//              query tile) into the 128-byte-swizzled K-major layout the
//              tensor core reads; a stage is handed over with an mbarrier
//              after the copies landed and a proxy fence (eight warps keep
//              enough 16-byte copies in flight for gathered rows);
//   warp 8     allocates 512 TMEM columns (two 128x256 fp32 accumulators)
//              and, from one lane, issues tcgen05.mma (K = 32 bytes each)
//              and the commits that free stages and publish accumulators;
//   warps 9-12 epilogue: tcgen05.ld of the accumulator rows (TMEM lane =
//              query), distance = ||q||^2 - 2 s_q s_x q.x + ||x||^2 (L2) or
//              -s_q s_x q.x (IP), predicate mask, and a per-query max-heap
//              of the k' best (key, id) composites in shared memory.
// The epilogue of tile t overlaps the MMAs of tile t+1 (double-buffered
// accumulators).  At the end each query's heap entries that beat the
// global per-query bound are appended to the candidate list.
//
// Every mbarrier wait is bounded; on timeout the kernel records an error
// in *err, lets copies and MMAs drain, frees its TMEM and returns.
#include <cudaTypedefs.h>

#include "topk_select.cuh"
#include "umma.cuh"
#include "vrs_internal.cuh"

namespace vrs {
namespace {

using namespace umma;

constexpr int kBM = 128;                 // queries per tile (TMEM lanes)
constexpr int kBN = 256;                 // rows per tile (accumulator columns)
constexpr int kBK = 128;                 // bytes of K per stage (one swizzle atom)
constexpr int kProdWarps = 8;           // gathered rows need many copies in flight
static_assert(256 * 8 % (32 * kProdWarps) == 0, "a stage's copies split evenly over the producers");
constexpr int kProdThreads = 32 * kProdWarps;
constexpr int kEpiThreads = 128;
constexpr int kMmaWarp = kProdWarps;
constexpr int kThreads = kProdThreads + 32 + kEpiThreads;
constexpr uint32_t kTmemCols = 512;
constexpr int kAStage = kBM * kBK;       // 16 KB
constexpr int kBStage = kBN * kBK;       // 32 KB

struct Layout {
    int nkb;        // K blocks of 128 bytes
    int ns;         // pipeline stages
    bool resa;      // queries resident for the whole kernel
    size_t a_off, b_off, bar_off, info_off, pid_off, ehist_off, heap_off, stash_off, total;
};

__host__ __device__ inline size_t al(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Capacity of a per-query global candidate buffer (room for one more
// 32-column chunk after a cut back to k').
__host__ __device__ inline int umma_bufcap(int kp) { return 2 * kp + 64; }

__host__ __device__ inline Layout make_layout(int row_bytes, int ns, bool resa, int kp_smem) {
    const int kp = kp_smem;   // 0 when the heaps live in global memory
    Layout L;
    L.nkb = (row_bytes + kBK - 1) / kBK;
    L.ns = ns;
    L.resa = resa;
    size_t off = 0;
    L.a_off = off;
    off += resa ? (size_t)L.nkb * kAStage : (size_t)ns * kAStage;
    L.b_off = off;
    off += (size_t)ns * kBStage;
    L.bar_off = off;
    off += al((2 * ns + 4 + 2) * 8 + 16, 16);   // full, empty, accfull x2, accempty x2, a_full, done, tmem, abort
    L.info_off = off;
    off += 2 * kBN * 12;                        // add f32, mul f32, id i32 per column, x2
    off += 2 * kMaxQCols * kBN * 4;             // per-query-predicate attribute values, x2
    L.pid_off = off;
    off += 2 * kBN * 4;                         // row ids of two tiles
    L.ehist_off = off;                          // radix-select histograms, 4 epilogue warps
    off += 4 * 256 * 4;
    off = al(off, 16);
    L.heap_off = off;
    off += (size_t)kp * kBM * 8;
    L.stash_off = off;                          // per-query stash of 16 candidates
    off += kp ? (size_t)16 * kBM * 8 : 0;
    L.total = off + 1024;                       // slack for 1024-byte alignment
    return L;
}

template <int DT>
__device__ __forceinline__ void issue_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    if constexpr (DT == 1) mma_f16(d, a, b, idesc(1, kBM, kBN), acc);
    else mma_f8(d, a, b, idesc(0, kBM, kBN), acc);
}

// Named barriers over a warp group, with an OR-reduction of a flag so that
// every thread of the group takes the same decision.
__device__ __forceinline__ bool bar_or(bool v, int id, int n) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ bool bar_epi_or(bool v) { return bar_or(v, 1, kEpiThreads); }
__device__ __forceinline__ bool bar_prod_or(bool v) { return bar_or(v, 2, kProdThreads); }

// Every lane waits; the warp agrees on the outcome.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
    const bool ok = mbar_wait(bar, parity, abort);
    return __all_sync(0xffffffffu, ok);
}

// DT: 1 = bf16 operands, 2 = FP8 E4M3 operands.  NS: pipeline stages.
template <int DT, int NS, bool RESA>
__global__ void __launch_bounds__(kThreads, 1)
umma_scan_kernel(const __grid_constant__ UmmaArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw_u32 = smem_u32(smem_raw);
    unsigned char *sm = smem_raw + (((raw_u32 + 1023u) & ~1023u) - raw_u32);
    const bool heap_smem = a.heap_g == nullptr;
    const Layout L = make_layout(a.row_bytes, NS, RESA, heap_smem ? a.kp : 0);
    unsigned char *Asm = sm + L.a_off;
    unsigned char *Bsm = sm + L.b_off;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L.bar_off);
    uint64_t *full = bars, *empty = bars + NS, *accfull = bars + 2 * NS,
             *accempty = bars + 2 * NS + 2, *a_full = bars + 2 * NS + 4, *done = bars + 2 * NS + 5;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * NS + 6);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    float *info_add = reinterpret_cast<float *>(sm + L.info_off);       // [2][kBN]
    float *info_mul = info_add + 2 * kBN;                                // [2][kBN]
    int32_t *info_id = reinterpret_cast<int32_t *>(info_mul + 2 * kBN);  // [2][kBN]
    int32_t *info_attr = info_id + 2 * kBN;                              // [2][kMaxQCols][kBN]
    int32_t *pid = reinterpret_cast<int32_t *>(sm + L.pid_off);          // [kBN]
    // heap_smem: [kp][kBM] per-query max-heaps in shared memory, interleaved
    // so a warp's accesses spread over the banks.  Otherwise each query has
    // an append-only candidate buffer of bufcap(kp) entries in global memory
    // (L2-resident), cut back to its k' best by a warp radix select when full.
    uint64_t *heap = heap_smem ? reinterpret_cast<uint64_t *>(sm + L.heap_off) : nullptr;
    uint64_t *stash = reinterpret_cast<uint64_t *>(sm + L.stash_off);   // [16][kBM]
    const int C = umma_bufcap(a.kp);
    int *ehist = reinterpret_cast<int *>(sm + L.ehist_off);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nqt = (a.B + kBM - 1) / kBM;
    const int qt = blockIdx.x % nqt, g = blockIdx.x / nqt, G = gridDim.x / nqt;
    const int64_t total = a.ids ? *a.count_dev : a.n_rows;
    const int64_t p0 = total * g / G, p1 = total * (g + 1) / G;
    const int T = (int)((p1 - p0 + kBN - 1) / kBN);
    const int nkb = L.nkb;
    const int kp = a.kp;

    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], kProdThreads);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accfull[i], 1);
            mbar_init(&accempty[i], kEpiThreads / 32);
        }
        mbar_init(a_full, kProdThreads);
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == kMmaWarp) {
        tmem_alloc(tmem_slot, kTmemCols);
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

    if (warp < kProdWarps) {
        // ------------------------------------------------------------ producers
        const int pt = tid;   // 0 .. kProdThreads - 1
        const unsigned char *Xb = a.X;
        const bool tma_x = a.use_tma_x && !a.ids;
        const bool tma_q = a.use_tma_q;
        if (RESA && tma_q) {
            if (pt == 0) {
                mbar_expect_tx(a_full, (uint32_t)(nkb * kAStage));
                for (int kb = 0; kb < nkb; ++kb)
                    tma_load_2d(smem_u32(Asm + (size_t)kb * kAStage), &a.tmQ, kb * kBK, qt * kBM,
                                a_full);
            }
            mbar_arrive(a_full);
        } else if (RESA) {
            for (int kb = 0; kb < nkb; ++kb)
                for (int idx = pt; idx < kBM * 8; idx += kProdThreads) {
                    const int r = idx >> 3, c = idx & 7;
                    const int off = kb * kBK + c * 16;
                    const uint32_t nb = off < a.row_bytes ? 16u : 0u;
                    const unsigned char *src = a.Q + ((int64_t)qt * kBM + r) * a.row_bytes + (nb ? off : 0);
                    cp_async16(smem_u32(Asm + (size_t)kb * kAStage + sw128_offset(r, c)), src, nb);
                }
            cp_async_commit();
            cp_async_wait<0>();
            fence_proxy_async_smem();
            mbar_arrive(a_full);
        }
        int it = 0;
        bool ok = true;
        // row ids of tile t (each producer one id of it; -1 past the range)
        auto id_of = [&](int t, int j) -> int32_t {
            const int64_t pos = p0 + (int64_t)t * kBN + j;
            return pos < p1 ? (a.ids ? a.ids[pos] : (int32_t)pos) : -1;
        };
        static_assert(kBN == kProdThreads, "one row id per producer thread");
        if (T > 0) pid[pt] = id_of(0, pt);
        for (int t = 0; t < T; ++t) {
            const int64_t pos0 = p0 + (int64_t)t * kBN;
            // this tile's ids are in place and the previous tile's reads of the
            // other buffer are done; stop together on failure
            if (bar_prod_or(!ok || *abort_flag)) break;
            const int32_t *pidt = pid + (t & 1) * kBN;
            // the next tile's id is loaded now and stored after this tile
            const int32_t nxt = t + 1 < T ? id_of(t + 1, pt) : -1;
            for (int kb = 0; kb < nkb; ++kb, ++it) {
                const int st = it % NS;
                if (!warp_wait(&empty[st], ((it / NS) & 1) ^ 1, abort_flag)) {
                    fail();
                    ok = false;
                    break;
                }
                unsigned char *bst = Bsm + (size_t)st * kBStage;
                if (pt == 0 && (tma_x || (!RESA && tma_q))) {
                    // TMA boxes: the stage's phase also waits for their bytes
                    mbar_expect_tx(&full[st], (uint32_t)((tma_x ? kBStage : 0) +
                                                         ((!RESA && tma_q) ? kAStage : 0)));
                    if (tma_x)
                        tma_load_2d(smem_u32(bst), &a.tmX, kb * kBK, (int32_t)pos0, &full[st]);
                    if (!RESA && tma_q)
                        tma_load_2d(smem_u32(Asm + (size_t)st * kAStage), &a.tmQ, kb * kBK,
                                    qt * kBM, &full[st]);
                }
                if (!tma_x) {
                    // the thread's row ids first, then its copies back to back
                    // (8 lanes copy one row's 128 bytes of this K block)
                    constexpr int kPer = kBN * 8 / kProdThreads;
                    int32_t rid[kPer];
#pragma unroll
                    for (int u = 0; u < kPer; ++u) rid[u] = pidt[(pt + u * kProdThreads) >> 3];
#pragma unroll
                    for (int u = 0; u < kPer; ++u) {
                        const int idx = pt + u * kProdThreads;
                        const int r = idx >> 3, c = idx & 7;
                        const int off = kb * kBK + c * 16;
                        const uint32_t nb = (rid[u] >= 0 && off < a.row_bytes) ? 16u : 0u;
                        const unsigned char *src = nb ? Xb + (int64_t)rid[u] * a.row_bytes + off : Xb;
                        cp_async16(smem_u32(bst + sw128_offset(r, c)), src, nb);
                    }
                }
                if (!RESA && !tma_q) {
                    unsigned char *ast = Asm + (size_t)st * kAStage;
                    for (int idx = pt; idx < kBM * 8; idx += kProdThreads) {
                        const int r = idx >> 3, c = idx & 7;
                        const int off = kb * kBK + c * 16;
                        const uint32_t nb = off < a.row_bytes ? 16u : 0u;
                        const unsigned char *src =
                            a.Q + ((int64_t)qt * kBM + r) * a.row_bytes + (nb ? off : 0);
                        cp_async16(smem_u32(ast + sw128_offset(r, c)), src, nb);
                    }
                }
                cp_async_commit();
                if (it >= NS - 1) {
                    cp_async_wait<NS - 1>();
                    fence_proxy_async_smem();
                    mbar_arrive(&full[(it - (NS - 1)) % NS]);
                }
            }
            pid[((t + 1) & 1) * kBN + pt] = nxt;   // (every producer is past tile t - 1)
        }
        // drain: the last min(it, NS-1) stages
        cp_async_wait<0>();
        fence_proxy_async_smem();
        for (int j = (it >= NS - 1 ? it - (NS - 1) : 0); j < it; ++j) mbar_arrive(&full[j % NS]);
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            bool ok = true;
            if (RESA && !mbar_wait(a_full, 0, abort_flag)) {
                fail();
                ok = false;
            }
            int it = 0;
            for (int t = 0; t < T && ok; ++t) {
                const int acc = t & 1, use = t >> 1;
                if (!mbar_wait(&accempty[acc], (use & 1) ^ 1, abort_flag)) {
                    fail();
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(acc * kBN);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int st = it % NS;
                    if (!mbar_wait(&full[st], (it / NS) & 1, abort_flag)) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t abase =
                        smem_u32(Asm + (size_t)(RESA ? kb : st) * kAStage);
                    const uint32_t bbase = smem_u32(Bsm + (size_t)st * kBStage);
#pragma unroll
                    for (int kk = 0; kk < kBK / 32; ++kk)
                        issue_mma<DT>(d, desc_sw128(abase + kk * 32), desc_sw128(bbase + kk * 32),
                                      (kb | kk) != 0 ? 1u : 0u);
                    mma_commit(&empty[st]);
                }
                if (!ok) break;
                mma_commit(&accfull[acc]);
            }
            // every MMA issued by this thread has completed once `done` flips
            mma_commit(done);
            if (!mbar_wait(done, 0, abort_flag)) {
                // the wait gave up because of an abort; wait again, bounded
                volatile int never = 0;
                mbar_wait(done, 0, &never);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int et = tid - (kProdThreads + 32);   // 0..127
        const int lq = warp & 3;                 // TMEM lane quarter of this warp
        const int qr = lq * 32 + lane;           // query row within the tile
        const int q = qt * kBM + qr;
        const bool qv = q < a.B;
        const float qn = (qv && a.metric == 0) ? a.qnorm[q] : 0.0f;
        const float qs = (qv && a.qscale) ? a.qscale[q] : 1.0f;
        const float mulc = a.metric == 0 ? -2.0f : -1.0f;
        // this query's own predicate (batched launch)
        int32_t qlo[kMaxQCols], qhi[kMaxQCols];
#pragma unroll
        for (int c = 0; c < kMaxQCols; ++c) {
            qlo[c] = (qv && c < a.nqc) ? a.qrange[((int64_t)q * a.nqc + c) * 2] : INT32_MIN;
            qhi[c] = (qv && c < a.nqc) ? a.qrange[((int64_t)q * a.nqc + c) * 2 + 1] : INT32_MAX;
        }
        const int nqc = a.nqc;
        // this query's own candidate width
        int kpq = kp;
        if (a.kq && qv) {
            const int kk = a.kq[q];
            kpq = max(kk * a.kp_factor, max(kk + 8, 8 * a.kp_factor));
            kpq = kpq < kp ? kpq : kp;
        }
        int hsize = 0;
        uint64_t tau = kEmpty, gcache = kEmpty, tcmp = kEmpty, published = kEmpty;
        auto H = [&](int i) -> uint64_t & { return heap[(size_t)i * kBM + qr]; };
        uint64_t *gbuf = heap_smem ? nullptr
                                   : a.heap_g + ((size_t)blockIdx.x * kBM + qr) * (size_t)C;
        int *wh = ehist + (warp - kMmaWarp - 1) * 256;
        // warp-cooperative cut of every lane whose buffer is about to fill (or
        // that can set its first bound); `final` cuts every buffer above k'
        auto warp_cuts = [&](bool final) {
            __syncwarp();
            unsigned need = __ballot_sync(0xffffffffu, qv && (final ? hsize > kpq
                                                                   : (hsize > C - 32 ||
                                                                      (tau == kEmpty && hsize >= kpq))));
            while (need) {
                const int l = __ffs(need) - 1;
                need &= need - 1;
                uint64_t *b = a.heap_g + ((size_t)blockIdx.x * kBM + lq * 32 + l) * (size_t)C;
                const int c = __shfl_sync(0xffffffffu, hsize, l);
                const int kl = __shfl_sync(0xffffffffu, kpq, l);
                const SelectResult sr = warp_select(b, c, kl, wh);
                uint64_t mx;
                const int kept = warp_pack(b, c, sr, &mx);
                if (lane == l) {
                    hsize = kept;
                    tau = mx;
                    tcmp = tau < gcache ? tau : gcache;
                }
            }
            __syncwarp();
        };
        // per-row values of a tile (norm, scale, id, this batch's predicate
        // columns) for the rows j = et and et + 128
        struct RowInfo {
            float add, mul;
            int32_t id;
            int32_t at[kMaxQCols];
        };
        RowInfo nxt[kBN / kEpiThreads];
        auto fetch_info = [&](int t, RowInfo (&ri)[kBN / kEpiThreads]) {
            const int64_t pos0 = p0 + (int64_t)t * kBN;
#pragma unroll
            for (int u = 0; u < kBN / kEpiThreads; ++u) {
                const int64_t pos = pos0 + et + u * kEpiThreads;
                bool okr = pos < p1;
                int32_t rid = -1;
                if (okr) {
                    rid = a.ids ? a.ids[pos] : (int32_t)pos;
                    if (!a.ids && a.bitmap) okr = (a.bitmap[rid >> 5] >> (rid & 31)) & 1u;
                }
                ri[u].add = okr ? (a.metric == 0 ? a.xnorm[rid] : 0.0f) : __int_as_float(0x7f800000);
                ri[u].mul = mulc * ((okr && a.xscale) ? a.xscale[rid] : 1.0f);
                ri[u].id = rid;
#pragma unroll
                for (int c = 0; c < kMaxQCols; ++c)
                    ri[u].at[c] = (okr && c < a.nqc) ? a.qcol[c][rid] : 0;
            }
        };
        auto store_info = [&](int acc, const RowInfo (&ri)[kBN / kEpiThreads]) {
#pragma unroll
            for (int u = 0; u < kBN / kEpiThreads; ++u) {
                const int j = et + u * kEpiThreads;
                info_add[acc * kBN + j] = ri[u].add;
                info_mul[acc * kBN + j] = ri[u].mul;
                info_id[acc * kBN + j] = ri[u].id;
#pragma unroll
                for (int c = 0; c < kMaxQCols; ++c)
                    if (c < a.nqc) info_attr[(acc * kMaxQCols + c) * kBN + j] = ri[u].at[c];
            }
        };
        if (T > 0) {
            fetch_info(0, nxt);
            store_info(0, nxt);
        }
        bool ok = true;
        for (int t = 0; t < T; ++t) {
            const int acc = t & 1, use = t >> 1;
            if (bar_epi_or(!ok || *abort_flag)) break;
            // the next tile's per-row values are loaded now and stored after
            // this tile, so their latency hides behind this tile's work
            if (t + 1 < T) fetch_info(t + 1, nxt);
            uint64_t gnext = kEmpty;
            if (qv) gnext = *reinterpret_cast<volatile uint64_t *>(a.tau_g + q);
            if (!warp_wait(&accfull[acc], use & 1, abort_flag)) {
                fail();
                ok = false;
                continue;
            }
            tc_fence_after();
            if (qv) {
                gcache = gnext;
                tcmp = tau < gcache ? tau : gcache;
            }
            const float *iadd = info_add + acc * kBN;
            const float *imul = info_mul + acc * kBN;
            const int32_t *iid = info_id + acc * kBN;
            const int32_t *iat = info_attr + acc * kMaxQCols * kBN;
            for (int ch = 0; ch < kBN / 32; ++ch) {
                uint32_t v[32];
                tmem_ld32(tmem_base + ((uint32_t)(lq * 32) << 16) + (uint32_t)(acc * kBN + ch * 32), v);
                tmem_ld_wait();
                if (!heap_smem) warp_cuts(false);
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    int ns = 0;   // stashed candidates of this half chunk
                    if (qv) {
                        const uint32_t thi = (uint32_t)(tcmp >> 32);
                        if (nqc) {
                            // per-query predicates: first every column's key and
                            // test (no branches, so the shared-memory loads of
                            // the 16 columns overlap), then the passing columns
                            const int j0 = ch * 32 + half * 16;
                            const float lo = a.metric == 0 ? 0.0f : -__int_as_float(0x7f800000);
                            const float tf = tcmp == kEmpty ? __int_as_float(0x7f800000)
                                                            : ordered_to_float(thi);
                            float key[16];
                            uint32_t pm = 0xffffu;
                            // this query's own ranges, 16 columns per 16-byte loads
#pragma unroll
                            for (int cc = 0; cc < kMaxQCols; ++cc) {
                                if (cc < nqc) {
#pragma unroll
                                    for (int c4 = 0; c4 < 4; ++c4) {
                                        const int4 av = *reinterpret_cast<const int4 *>(iat + cc * kBN + j0 + 4 * c4);
                                        const int32_t avs[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
                                        for (int u = 0; u < 4; ++u)
                                            if (!(avs[u] >= qlo[cc] && avs[u] <= qhi[cc])) pm &= ~(1u << (4 * c4 + u));
                                    }
                                }
                            }
#pragma unroll
                            for (int c4 = 0; c4 < 4; ++c4) {
                                const float4 x = *reinterpret_cast<const float4 *>(iadd + j0 + 4 * c4);
                                const float4 y = *reinterpret_cast<const float4 *>(imul + j0 + 4 * c4);
                                const float ad[4] = {x.x, x.y, x.z, x.w}, mu[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
                                for (int u = 0; u < 4; ++u) {
                                    const int c = 4 * c4 + u;
                                    const float kk = fmaxf(fmaf(__uint_as_float(v[half * 16 + c]) * qs, mu[u], qn + ad[u]), lo);
                                    key[c] = kk;
                                    if (!(kk <= tf && kk < __int_as_float(0x7f800000))) pm &= ~(1u << c);
                                }
                            }
                            if (pm) {
#pragma unroll
                                for (int c = 0; c < 16; ++c) {
                                    if (!((pm >> c) & 1u)) continue;
                                    const uint64_t cd = make_cand(key[c], iid[j0 + c]);
                                    if (cd < tcmp) {
                                        if (heap_smem) stash[(size_t)(ns++) * kBM + qr] = cd;
                                        else gbuf[hsize++] = cd;
                                    }
                                }
                            }
                        } else {
                            // shared predicate (or none): the 16 columns' norms
                            // and scales with 16-byte loads, every key and its
                            // test against the bound as a float (no branch),
                            // then the passing columns one by one
                            const int j0 = ch * 32 + half * 16;
                            float ad[16], mu[16];
#pragma unroll
                            for (int c4 = 0; c4 < 4; ++c4) {
                                const float4 x = *reinterpret_cast<const float4 *>(iadd + j0 + 4 * c4);
                                const float4 y = *reinterpret_cast<const float4 *>(imul + j0 + 4 * c4);
                                ad[4 * c4] = x.x; ad[4 * c4 + 1] = x.y; ad[4 * c4 + 2] = x.z; ad[4 * c4 + 3] = x.w;
                                mu[4 * c4] = y.x; mu[4 * c4 + 1] = y.y; mu[4 * c4 + 2] = y.z; mu[4 * c4 + 3] = y.w;
                            }
                            const float lo = a.metric == 0 ? 0.0f : -__int_as_float(0x7f800000);
                            // keys above the bound's key fail (ties go on to the
                            // composite test below)
                            const float tf = tcmp == kEmpty ? __int_as_float(0x7f800000)
                                                            : ordered_to_float(thi);
                            float key[16];
                            uint32_t pm = 0;
#pragma unroll
                            for (int c = 0; c < 16; ++c) {
                                const float kk = fmaxf(fmaf(__uint_as_float(v[half * 16 + c]) * qs, mu[c], qn + ad[c]), lo);
                                key[c] = kk;
                                pm |= (uint32_t)(kk <= tf && kk < __int_as_float(0x7f800000)) << c;
                            }
                            if (pm) {
#pragma unroll
                                for (int c = 0; c < 16; ++c) {
                                    if (!((pm >> c) & 1u)) continue;
                                    const uint64_t cd = make_cand(key[c], iid[j0 + c]);
                                    if (cd < tcmp) {
                                        if (heap_smem) stash[(size_t)(ns++) * kBM + qr] = cd;
                                        else gbuf[hsize++] = cd;
                                    }
                                }
                            }
                        }
                    }
                    if (!heap_smem) continue;
                    // insert the stashed candidates: the lanes of a warp run
                    // these loops together, one round per stashed entry
                    for (int i = 0; i < ns; ++i) {
                        const uint64_t cd = stash[(size_t)i * kBM + qr];
                        if (cd >= tcmp) continue;
                        if (hsize < kpq) {
                            H(hsize++) = cd;
                            if (hsize == kpq) {
                                // bottom-up heap construction once k' are in
                                for (int r0 = kpq / 2 - 1; r0 >= 0; --r0) {
                                    const uint64_t x = H(r0);
                                    int h = r0;
                                    while (true) {
                                        const int l = 2 * h + 1;
                                        if (l >= kpq) break;
                                        const int r = l + 1;
                                        const int m = (r < kpq && H(r) > H(l)) ? r : l;
                                        const uint64_t hm = H(m);
                                        if (hm <= x) break;
                                        H(h) = hm;
                                        h = m;
                                    }
                                    H(h) = x;
                                }
                                tau = H(0);
                            }
                        } else {
                            int h = 0;
                            while (true) {
                                const int l = 2 * h + 1;
                                if (l >= kpq) break;
                                const int r = l + 1;
                                const int m = (r < kpq && H(r) > H(l)) ? r : l;
                                const uint64_t hm = H(m);
                                if (hm <= cd) break;
                                H(h) = hm;
                                h = m;
                            }
                            H(h) = cd;
                            tau = H(0);
                        }
                        tcmp = tau < gcache ? tau : gcache;
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty[acc]);
            if (t + 1 < T) store_info(acc ^ 1, nxt);
            // publish this query's bound only when it improved since the last
            // publication and beats the one already known
            if (qv && tau < published && tau < gcache) {
                atomicMin(reinterpret_cast<unsigned long long *>(a.tau_g + q),
                          (unsigned long long)tau);
                published = tau;
            }
        }
        // append the entries that beat the global bound
        if (!heap_smem && ok) {
            warp_cuts(true);
            if (qv && hsize == kpq && tau == kEmpty) {
                uint64_t mx = 0;
                for (int i = 0; i < hsize; ++i) mx = gbuf[i] > mx ? gbuf[i] : mx;
                tau = mx;
            }
            if (qv && tau != kEmpty && hsize >= kpq)
                atomicMin(reinterpret_cast<unsigned long long *>(a.tau_g + q),
                          (unsigned long long)tau);
        }
        if (qv) {
            const uint64_t gb = *reinterpret_cast<volatile uint64_t *>(a.tau_g + q);
            auto E = [&](int i) -> uint64_t { return heap_smem ? H(i) : gbuf[i]; };
            int n_out = 0;
            for (int i = 0; i < hsize; ++i) n_out += E(i) <= gb;
            if (n_out) {
                int pos = atomicAdd(a.out_cnt + q, n_out);
                uint64_t *o = a.out + (int64_t)q * a.out_cap;
                // the list holds every CTA's heap; past its end nothing is
                // written and the error word says so
                if (pos + n_out > a.out_cap) atomicExch(a.err, 2);
                for (int i = 0; i < hsize; ++i)
                    if (E(i) <= gb) {
                        if (pos < a.out_cap) o[pos] = E(i);
                        ++pos;
                    }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

template <int DT, int NS, bool RESA>
cudaError_t launch_t(const UmmaArgs &a, int grid, size_t smem, cudaStream_t s) {
    auto k = umma_scan_kernel<DT, NS, RESA>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

constexpr size_t kSmemMax = 227 * 1024;

// Chooses stages, resident queries and the heap location for the shared-
// memory budget: heaps in shared memory when they fit next to >= 3 stages
// (or 2 with resident queries), else in global memory (L2-resident).
bool umma_config(int row_bytes, int kp, int *ns, bool *resa, size_t *smem, bool *heap_in_smem) {
    for (int hs = 1; hs >= 0; --hs) {
        for (int pass = 0; pass < 2; ++pass) {
            const bool r = pass == 0;
            for (int n = 4; n >= (hs ? 3 : 2); --n) {
                Layout L = make_layout(row_bytes, n, r, hs ? kp : 0);
                if (L.total <= kSmemMax) {
                    *ns = n;
                    *resa = r;
                    *smem = L.total;
                    *heap_in_smem = hs != 0;
                    return true;
                }
            }
        }
    }
    return false;
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
}

bool make_tmap_2d(CUtensorMap *m, const void *base, uint64_t inner_bytes, uint64_t rows,
                  uint32_t box_rows) {
    if (!g_encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return false;
        }
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    if (inner_bytes < kBK || inner_bytes % 16 || reinterpret_cast<uintptr_t>(base) % 16) return false;
    const cuuint64_t dims[2] = {inner_bytes, rows};
    const cuuint64_t strides[1] = {inner_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, box_rows};
    const cuuint32_t es[2] = {1, 1};
    return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides,
                    box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t umma_global_buffer_bytes(int grid, int kp) {
    return (size_t)grid * kBM * umma_bufcap(kp) * 8;
}

cudaError_t launch_umma(const UmmaArgs &a, int dtype, int grid, cudaStream_t s) {
    int ns;
    bool resa, hs;
    size_t smem;
    if (!umma_config(a.row_bytes, a.kp, &ns, &resa, &smem, &hs) || a.err == nullptr)
        return cudaErrorInvalidValue;
    if (!hs && a.heap_g == nullptr) return cudaErrorInvalidValue;
    if (hs && a.heap_g != nullptr) return cudaErrorInvalidValue;
#define VRS_CASE(DT, NS, RA)                                        \
    if (dtype == DT && ns == NS && resa == RA) return launch_t<DT, NS, RA>(a, grid, smem, s);
    VRS_CASE(1, 4, true) VRS_CASE(1, 3, true) VRS_CASE(1, 2, true)
    VRS_CASE(1, 4, false) VRS_CASE(1, 3, false) VRS_CASE(1, 2, false)
    VRS_CASE(2, 4, true) VRS_CASE(2, 3, true) VRS_CASE(2, 2, true)
    VRS_CASE(2, 4, false) VRS_CASE(2, 3, false) VRS_CASE(2, 2, false)
#undef VRS_CASE
    return cudaErrorInvalidValue;
}

}  // namespace vrs
