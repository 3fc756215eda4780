// k_umma_pair.cu -- the dense-key distance pass for float32 rows and small
// query batches on the tensor cores, reading a load-time bf16 pair copy.
//
// Each float32 value is stored once more at load as two bf16 parts,
// x = x1 + x2 + e with x1 = bf16(x), x2 = bf16(x - x1) and |e| <= 2^-16 |x|
// (the same 4 bytes per element as the float32 row, so the gather moves no
// more bytes).  Queries get the same split at query time.  The pass forms
//     q.x ~= q1.x1 + q1.x2 + q2.x1
// with bf16 operands (kind::f16, FP32 accumulation in tensor memory): each
// product of bf16 values is exact in FP32, the dropped q2.x2 and the residuals
// leave a few 2^-16 relative per product, and the exact FP32 re-rank with the
// certificate decides the result (CertArgs, the BF16x3 family).
//
// Rows are the MMA's M dimension (128 selected rows per tile), queries its N
// (2 NQ columns: [q1 ; q2]).  A pair row holds [x1 (ldp values) | x2 (ldp
// values)], ldp = round_up(d, 64), so its 128-byte K blocks are first the x1
// blocks, then the x2 blocks; an x1 block multiplies the [q1 ; q2] block of the
// same dimensions (N = 2 NQ), an x2 block multiplies q1 alone (N = NQ), and the
// epilogue adds column j and column NQ + j.
//
// Warp roles (288 threads):
//   warps 0-3  producers: the row ids of up to kIdTiles tiles go to shared
//              memory; then a stage of KBS K blocks of a tile (KBS = 4, or 2
//              when the blocks of a row do not split into fours) is gathered
//              with 16-byte cp.async copies straight into the 128-byte-
//              swizzled K-major layout the tensor core reads.  The lanes of a
//              warp copy KBS x 128 contiguous bytes of each row they take (a
//              whole 512-byte row at d = 128), so every row is read in one
//              piece.  Stages of 32-64 KB in a ring of 2-3 keep up to ~190 KB
//              per SM in flight; a stage is handed over after its copies
//              landed and a proxy fence;
//   warp 4     allocates TMEM and, from one lane, issues tcgen05.mma and the
//              commits that free stages and publish accumulators
//              (double-buffered);
//   warps 5-8  epilogue: tcgen05.ld of a row's 2 NQ accumulator columns, the
//              keys written to the dense key matrix, and each query's minimum
//              over the tile (one 128-position chunk).
// Every mbarrier wait is bounded; on timeout the kernel records an error in
// *err, lets the copies and MMAs drain, frees its TMEM and returns.
#include <algorithm>

#include "umma.cuh"
#include "vrs_internal.cuh"

namespace vrs {
namespace {

using namespace umma;

constexpr int kM = 128;                  // rows per tile (TMEM lanes)
constexpr int kBK = 128;                 // bytes of K per stage (one swizzle atom)
constexpr int kProdWarps = 8;
constexpr int kProdThreads = kProdWarps * 32;
constexpr int kKB = kM * kBK;            // 16 KB: one K block of a tile
constexpr int kIdTiles = 16;             // tiles whose row ids are staged at a time
// EG epilogue warps per TMEM lane quarter (each takes NQ / EG queries)
__host__ __device__ constexpr int epi_threads(int eg) { return 128 * eg; }
__host__ __device__ constexpr int all_threads(int eg) { return kProdThreads + 32 + 128 * eg; }
// epilogue warps per lane quarter for NQ queries per tile
__host__ __device__ constexpr int pair_eg(int nq) { return nq <= 16 ? 2 : 4; }

struct PLayout {
    int nkb, nkbh, kbs;   // K blocks per row, per part, per stage
    size_t b_off, a_off, bar_off, qn_off, sid_off, total;
};

__host__ __device__ inline size_t pal(size_t x, size_t a) { return (x + a - 1) / a * a; }

// K blocks per stage: 4 when a row's blocks split into fours, else 2
__host__ __device__ inline int pair_kbs(int ldp) { return (2 * (ldp / 64)) % 4 == 0 ? 4 : 2; }

// ldp: elements per part of a pair row (a multiple of 64)
__host__ __device__ inline PLayout playout(int ldp, int nq, int ns) {
    PLayout L;
    L.nkbh = ldp / 64;                            // K blocks per part
    L.nkb = 2 * L.nkbh;
    L.kbs = pair_kbs(ldp);
    size_t o = 0;
    L.b_off = o;                                  // [nkbh][2 nq rows x 128 B]
    o += (size_t)L.nkbh * 2 * nq * kBK;
    o = pal(o, 1024);
    L.a_off = o;                                  // [ns][kbs][128 rows x 128 B]
    o += (size_t)ns * L.kbs * kKB;
    L.bar_off = o;                                // full, empty, accfull x2, accempty x2, done
    o += pal((size_t)(2 * ns + 5) * 8 + 16, 16);
    L.qn_off = o;
    o += pal((size_t)nq * 4, 16);
    L.sid_off = o;
    o += (size_t)kIdTiles * kM * 4;
    L.total = o + 1024;                           // slack for 1024-byte alignment
    return L;
}

__host__ __device__ constexpr uint32_t pair_tmem_cols(int nq) {
    return 4 * nq <= 32 ? 32u : 4 * nq <= 64 ? 64u : 4 * nq <= 128 ? 128u : 256u;
}

template <int N>
__device__ __forceinline__ bool epi_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(N)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ bool prod_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 2, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kProdThreads)
        : "memory");
    return r != 0;
}
template <int N>
__device__ __forceinline__ void builders_sync() {
    asm volatile("bar.sync 3, %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
    return __all_sync(0xffffffffu, mbar_wait(bar, parity, abort));
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}

template <int NQ, int NS, int KBS, int EG>
__global__ void __launch_bounds__(all_threads(EG), 1)
umma_pair_kernel(ScanArgs a, const unsigned char *__restrict__ Xp, int ldp) {
    constexpr int QG = NQ / EG;                         // queries per epilogue warp
    constexpr int kEpiThreads = epi_threads(EG);
    constexpr int kThreads = all_threads(EG);
    constexpr int kBuilders = kThreads - kProdThreads;  // MMA + epilogue threads
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw_u32 = smem_u32(smem_raw);
    unsigned char *sm = smem_raw + (((raw_u32 + 1023u) & ~1023u) - raw_u32);
    const int row_bytes = 4 * ldp;
    const PLayout L = playout(ldp, NQ, NS);
    const int nkb = L.nkb, nkbh = L.nkbh, nst = nkb / KBS;   // stages per tile
    constexpr int kbs = KBS;
    constexpr size_t stage_bytes = (size_t)KBS * kKB;
    unsigned char *Bsm = sm + L.b_off;
    unsigned char *Asm = sm + L.a_off;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L.bar_off);
    uint64_t *full = bars, *empty = bars + NS, *accfull = bars + 2 * NS,
             *accempty = bars + 2 * NS + 2, *done = bars + 2 * NS + 4;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * NS + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    float *qn = reinterpret_cast<float *>(sm + L.qn_off);
    int32_t *sid = reinterpret_cast<int32_t *>(sm + L.sid_off);
    __shared__ uint32_t cmin_s[2][4][NQ];   // per tile: each lane quarter's minimum per query
    constexpr uint32_t kCols = pair_tmem_cols(NQ);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nqt = (a.B + NQ - 1) / NQ;
    const int qt = blockIdx.x % nqt, g = blockIdx.x / nqt, G = gridDim.x / nqt;
    const int q0 = qt * NQ;
    // a programmatic dependent of the filter kernel: the set-up below
    // overlaps its tail; the selected-row count and ids are read after the wait
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], kProdThreads);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accfull[i], 1);
            mbar_init(&accempty[i], kEpiThreads / 32);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == kProdWarps) {
        tmem_alloc(tmem_slot, kCols);
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

    if (warp >= kProdWarps) {
        // MMA and epilogue warps build the B operand: K block kb (dimensions
        // 64 kb .. 64 kb + 63) holds [q1 ; q2] of this CTA's queries (zero past
        // B and past d), 128-byte-swizzled K-major; and ||q||^2 in float32
        const int bt = tid - kProdThreads;
        for (int idx = bt; idx < nkbh * 2 * NQ * 8; idx += kBuilders) {
            const int c = idx & 7, r = (idx >> 3) % (2 * NQ), kb = (idx >> 3) / (2 * NQ);
            const int j = r % NQ, t0 = kb * 64 + c * 8;
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int t = t0 + u;
                v[u] = (q0 + j < a.B && t < a.d) ? a.Q[(int64_t)(q0 + j) * a.ld + t] : 0.0f;
                if (r >= NQ) v[u] -= __bfloat162float(__float2bfloat16_rn(v[u]));
            }
            uint4 o;
            o.x = pack_bf16(v[0], v[1]);
            o.y = pack_bf16(v[2], v[3]);
            o.z = pack_bf16(v[4], v[5]);
            o.w = pack_bf16(v[6], v[7]);
            *reinterpret_cast<uint4 *>(Bsm + (size_t)kb * 2 * NQ * kBK + sw128_offset(r, c)) = o;
        }
        for (int j = warp - kProdWarps; j < NQ; j += kBuilders / 32) {
            float s2 = 0.0f;
            if (q0 + j < a.B)
                for (int t = lane; t < a.d; t += 32) {
                    const float v = a.Q[(int64_t)(q0 + j) * a.ld + t];
                    s2 = fmaf(v, v, s2);
                }
            for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            if (lane == 0) qn[j] = s2;
        }
        fence_proxy_async_smem();
        builders_sync<kBuilders>();
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int64_t total = *a.count_dev;
    if (a.count_copy && blockIdx.x == 0 && tid == 0) *a.count_copy = total;
    const int64_t nch = (total + kM - 1) / kM;
    const int64_t c0 = nch * g / G, c1 = nch * (g + 1) / G;
    const int T = (int)(c1 - c0);

    if (warp < kProdWarps) {
        // ------------------------------------------------------------ producers
        // lane l copies 16-byte chunk (l & 7) of the stage's K block
        // (l >> 3) % KBS of its rows, so 8 KBS lanes read 128 KBS contiguous
        // bytes of one row; warp w takes rows w + kProdWarps j.  Each thread
        // reads its row ids for a stage first and then issues its copies, all
        // unrolled, so the copies leave back to back.
        constexpr int kLpr = 8 * KBS;                      // lanes per row
        constexpr int kRpi = 32 / kLpr;                    // rows per warp instruction
        constexpr int kIter = kM / (kProdWarps * kRpi);    // copies per thread per stage
        constexpr int kSid = kIdTiles * kM / kProdThreads; // staged ids per thread
        const int cc = lane & 7, kbl = (lane >> 3) % KBS, rl = lane / kLpr;
        int it = 0;
        bool ok = true;
        for (int sc = 0; sc < T && ok; sc += kIdTiles) {
            const int nt = min(kIdTiles, T - sc);
            if (prod_or(false)) break;   // every producer is done with the previous ids
            const int64_t pbase = (c0 + sc) * kM;
            {
                int32_t v[kSid];
#pragma unroll
                for (int u = 0; u < kSid; ++u) {
                    const int i = tid + u * kProdThreads;
                    v[u] = (i < nt * kM && pbase + i < total) ? a.ids[pbase + i] : -1;
                }
#pragma unroll
                for (int u = 0; u < kSid; ++u) sid[tid + u * kProdThreads] = v[u];
            }
            if (prod_or(false)) break;
            for (int tt = 0; tt < nt && ok; ++tt) {
                for (int sg = 0; sg < nst; ++sg, ++it) {
                    const int st = it % NS;
                    if (!warp_wait(&empty[st], ((it / NS) & 1) ^ 1, abort_flag)) {
                        if (lane == 0) fail();
                        ok = false;
                        break;
                    }
                    const int kb = sg * KBS + kbl;
                    const uint32_t dst = smem_u32(Asm + (size_t)st * stage_bytes + (size_t)kbl * kKB);
                    int32_t rid[kIter];
#pragma unroll
                    for (int i = 0; i < kIter; ++i)
                        rid[i] = sid[tt * kM + warp + kProdWarps * (i * kRpi + rl)];
#pragma unroll
                    for (int i = 0; i < kIter; ++i) {
                        const int r = warp + kProdWarps * (i * kRpi + rl);
                        const unsigned char *src =
                            rid[i] >= 0 ? Xp + (int64_t)rid[i] * row_bytes + kb * kBK + cc * 16 : Xp;
                        cp_async16(dst + sw128_offset(r, cc), src, rid[i] >= 0 ? 16u : 0u);
                    }
                    cp_async_commit();
                    if (it >= NS - 1) {
                        cp_async_wait<NS - 1>();
                        fence_proxy_async_smem();
                        mbar_arrive(&full[(it - (NS - 1)) % NS]);
                    }
                }
            }
            ok = !prod_or(!ok);
        }
        // drain: the last min(it, NS - 1) stages
        cp_async_wait<0>();
        fence_proxy_async_smem();
        for (int j = (it >= NS - 1 ? it - (NS - 1) : 0); j < it; ++j) mbar_arrive(&full[j % NS]);
    } else if (warp == kProdWarps) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t id_full = idesc(1, kM, 2 * NQ), id_half = idesc(1, kM, NQ);
            const uint32_t bbase = smem_u32(Bsm);
            int s = 0;
            bool ok = true;
            // test hook: phase 0 of `done` completes only at this thread's
            // final commit, so waiting for it here runs out the bounded wait
            // (~1 s) and the kernel takes its failure path: error word,
            // abort, drain, TMEM freed
            if (a.wait_test && !mbar_wait(done, 0, abort_flag)) {
                fail();
                ok = false;
            }
            for (int t = 0; t < T && ok; ++t) {
                const int acc = t & 1, use = t >> 1;
                if (!mbar_wait(&accempty[acc], (use & 1) ^ 1, abort_flag)) {
                    fail();
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(acc * 2 * NQ);
                for (int sg = 0; sg < nst; ++sg, ++s) {
                    const int st = s % NS;
                    if (!mbar_wait(&full[st], (s / NS) & 1, abort_flag)) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int kbl = 0; kbl < kbs; ++kbl) {
                        const int kb = sg * kbs + kbl;
                        const uint32_t abase = smem_u32(Asm + (size_t)st * stage_bytes + (size_t)kbl * kKB);
                        const bool hi = kb < nkbh;
                        const uint32_t bk = bbase + (uint32_t)((hi ? kb : kb - nkbh) * 2 * NQ * kBK);
#pragma unroll
                        for (int kk = 0; kk < kBK / 32; ++kk)
                            mma_f16(d, desc_sw128(abase + kk * 32), desc_sw128(bk + kk * 32),
                                    hi ? id_full : id_half, (kb | kk) != 0 ? 1u : 0u);
                    }
                    mma_commit(&empty[st]);
                }
                if (!ok) break;
                mma_commit(&accfull[acc]);
            }
            // every MMA issued by this thread has completed once `done` flips
            mma_commit(done);
            if (!mbar_wait(done, 0, abort_flag)) {
                volatile int never = 0;
                mbar_wait(done, 0, &never);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        // warp (quarter lq, group eg) reads TMEM lanes 32 lq .. 32 lq + 31 (its
        // rows) and takes queries eg QG .. eg QG + QG - 1
        const int ew = warp - kProdWarps - 1;    // 0 .. 4 EG - 1
        const int lq = warp & 3;                 // TMEM lane quarter (warp id mod 4)
        const int eg = ew / 4;                   // query group of this warp
        const int jb = eg * QG;                  // its first query
        const int row = lq * 32 + lane;          // row within the tile
        const float mulc = a.metric == 0 ? -2.0f : -1.0f;
        float qnr[QG];
#pragma unroll
        for (int j = 0; j < QG; ++j) qnr[j] = qn[jb + j];
        auto valid_at = [&](int t) { return t < T && (c0 + t) * kM + row < total; };
        auto id_at = [&](int t) -> int32_t { return valid_at(t) ? a.ids[(c0 + t) * kM + row] : 0; };
        auto xn_of = [&](int t, int32_t id) -> float {
            return (valid_at(t) && a.metric == 0) ? __ldg(a.xnorm + id) : 0.0f;
        };
        // row ids four tiles ahead and norms two tiles ahead (a shift
        // register), so the key of a tile does not wait on loaded DRAM latency
        int32_t id2 = id_at(2), id3 = id_at(3), id4 = id_at(4);
        float xn0 = xn_of(0, id_at(0)), xn1 = xn_of(1, id_at(1));
        for (int t = 0; t < T; ++t) {
            const int acc = t & 1, use = t >> 1;
            const int64_t pos = (c0 + t) * kM + row;
            const bool valid = pos < total;
            const float xn = xn0;
            xn0 = xn1;
            xn1 = xn_of(t + 2, id2);
            id2 = id3;
            id3 = id4;
            id4 = id_at(t + 5);
            const bool okw = warp_wait(&accfull[acc], use & 1, abort_flag);
            if (epi_or<kEpiThreads>(!okw)) {
                if (!okw && lane == 0) fail();
                break;
            }
            tc_fence_after();
            const uint32_t tbase = tmem_base + ((uint32_t)(lq * 32) << 16) + (uint32_t)(acc * 2 * NQ);
            // columns [jb, jb + QG): q1.x1 + q1.x2; [NQ + jb, NQ + jb + QG): q2.x1
            float key[QG];
            {
                uint32_t va[QG], vb[QG];
                tmem_ldn<QG>(tbase + jb, va);
                tmem_ldn<QG>(tbase + NQ + jb, vb);
                tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < QG; ++j) key[j] = __uint_as_float(va[j]) + __uint_as_float(vb[j]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty[acc]);
            const int buf = t & 1;
            float *kp = a.keys_out + (int64_t)(q0 + jb) * a.keys_ld + pos;
#pragma unroll
            for (int j = 0; j < QG; ++j) {
                const float k = a.metric == 0 ? fmaxf(fmaf(mulc, key[j], qnr[j] + xn), 0.0f) : -key[j];
                const bool w = valid && q0 + jb + j < a.B;
                if (w) kp[(int64_t)j * a.keys_ld] = k;
                const uint32_t m = __reduce_min_sync(0xffffffffu, w ? float_to_ordered(k) : 0xffffffffu);
                if (lane == j) cmin_s[buf][lq][jb + j] = m;
            }
            epi_or<kEpiThreads>(false);
            const int et = tid - (kProdThreads + 32);
            if (et < NQ && q0 + et < a.B) {
                const uint32_t m = min(min(cmin_s[buf][0][et], cmin_s[buf][1][et]),
                                       min(cmin_s[buf][2][et], cmin_s[buf][3][et]));
                a.chunk_min[(int64_t)(q0 + et) * a.cmin_ld + c0 + t] = m;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == kProdWarps) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kCols);
    }
}

// query tile: 16 or 32 queries (larger batches take several tiles; a 64-query
// tile is epilogue-bound)
int pair_nq(int B) { return B <= 16 ? 16 : 32; }

// Stages that fit next to the B operand (3 or 2, or 4 of 32 KB).
int pair_stages(int ldp, int nq) {
    for (int ns : {4, 3, 2}) {
        if (ns == 4 && pair_kbs(ldp) != 2) continue;
        if (playout(ldp, nq, ns).total <= (size_t)227 * 1024) return ns;
    }
    return 0;
}

template <int NQ, int NS, int KBS>
cudaError_t launch_t(const ScanArgs &a, const unsigned char *Xp, int ldp, int G, cudaStream_t s) {
    constexpr int EG = pair_eg(NQ);
    const size_t sm = playout(ldp, NQ, NS).total;
    cudaError_t e = cudaFuncSetAttribute(umma_pair_kernel<NQ, NS, KBS, EG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int nqt = (a.B + NQ - 1) / NQ;
    return launch_dependent(umma_pair_kernel<NQ, NS, KBS, EG>, dim3(nqt * G),
                            dim3(all_threads(EG)), sm, s, a, Xp, ldp);
}

template <int NQ>
cudaError_t launch_nq(const ScanArgs &a, const unsigned char *Xp, int ldp, int G, int ns,
                      cudaStream_t s) {
    if (pair_kbs(ldp) == 4) return ns == 3 ? launch_t<NQ, 3, 4>(a, Xp, ldp, G, s)
                                           : launch_t<NQ, 2, 4>(a, Xp, ldp, G, s);
    switch (ns) {
        case 4: return launch_t<NQ, 4, 2>(a, Xp, ldp, G, s);
        case 3: return launch_t<NQ, 3, 2>(a, Xp, ldp, G, s);
        default: return launch_t<NQ, 2, 2>(a, Xp, ldp, G, s);
    }
}

}  // namespace

int pair_ld(int d) { return (d + 63) / 64 * 64; }

bool umma_pair_fits(int B, int d) { return B <= 64 && pair_stages(pair_ld(d), pair_nq(B)) > 0; }

int umma_pair_grid(int B, int n_sm) {
    const int nqt = (B + pair_nq(B) - 1) / pair_nq(B);
    return std::max(1, n_sm / nqt);
}

cudaError_t launch_umma_pair(const ScanArgs &a, const void *Xp, int G, cudaStream_t s) {
    const int ldp = pair_ld(a.d);
    const int nq = pair_nq(a.B);
    const int ns = pair_stages(ldp, nq);
    if (ns == 0 || a.B > 64 || !Xp || a.keys_out == nullptr || a.ids == nullptr ||
        a.count_dev == nullptr || a.chunk_min == nullptr || a.err == nullptr ||
        reinterpret_cast<uintptr_t>(Xp) % 16)
        return cudaErrorInvalidValue;
    const unsigned char *xp = static_cast<const unsigned char *>(Xp);
    return nq == 16 ? launch_nq<16>(a, xp, ldp, G, ns, s) : launch_nq<32>(a, xp, ldp, G, ns, s);
}

}  // namespace vrs
