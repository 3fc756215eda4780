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
constexpr int kProdWarps = 4;
constexpr int kProdThreads = kProdWarps * 32;
constexpr int kEpiThreads = 128;
constexpr int kThreads = kProdThreads + 32 + kEpiThreads;   // 288
constexpr int kKB = kM * kBK;            // 16 KB: one K block of a tile
constexpr int kIdTiles = 16;             // tiles whose row ids are staged at a time
constexpr int kBuilders = kThreads - kProdThreads;   // MMA + epilogue threads: 160

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

__device__ __forceinline__ bool epi_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kEpiThreads)
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
__device__ __forceinline__ void builders_sync() {
    asm volatile("bar.sync 3, %0;" ::"n"(kBuilders) : "memory");
}
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
    return __all_sync(0xffffffffu, mbar_wait(bar, parity, abort));
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}

template <int NQ, int NS>
__global__ void __launch_bounds__(kThreads, 1)
umma_pair_kernel(ScanArgs a, const unsigned char *__restrict__ Xp, int ldp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw_u32 = smem_u32(smem_raw);
    unsigned char *sm = smem_raw + (((raw_u32 + 1023u) & ~1023u) - raw_u32);
    const int row_bytes = 4 * ldp;
    const PLayout L = playout(ldp, NQ, NS);
    const int nkb = L.nkb, nkbh = L.nkbh, kbs = L.kbs, nst = nkb / kbs;   // stages per tile
    const size_t stage_bytes = (size_t)kbs * kKB;
    unsigned char *Bsm = sm + L.b_off;
    unsigned char *Asm = sm + L.a_off;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L.bar_off);
    uint64_t *full = bars, *empty = bars + NS, *accfull = bars + 2 * NS,
             *accempty = bars + 2 * NS + 2, *done = bars + 2 * NS + 4;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * NS + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    float *qn = reinterpret_cast<float *>(sm + L.qn_off);
    int32_t *sid = reinterpret_cast<int32_t *>(sm + L.sid_off);
    __shared__ uint32_t cmin_s[2][NQ];
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
    for (int j = tid; j < 2 * NQ; j += kThreads) cmin_s[j / NQ][j % NQ] = 0xffffffffu;
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
        builders_sync();
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int64_t total = *a.count_dev;
    const int64_t nch = (total + kM - 1) / kM;
    const int64_t c0 = nch * g / G, c1 = nch * (g + 1) / G;
    const int T = (int)(c1 - c0);

    if (warp < kProdWarps) {
        // ------------------------------------------------------------ producers
        // warp w takes rows w + 4 j of the tile; lane l copies 16-byte chunk
        // (l & 7) of the stage's K block (l >> 3) % kbs of row
        // w + 4 (i (32 / (8 kbs)) + l / (8 kbs)), so 8 kbs lanes read 128 kbs
        // contiguous bytes of one row
        const int lpr = 8 * kbs;            // lanes per row
        const int rpi = 32 / lpr;           // rows per warp instruction
        const int cc = lane & 7, kbl = (lane >> 3) % kbs, rl = lane / lpr;
        int it = 0;
        bool ok = true;
        for (int sc = 0; sc < T && ok; sc += kIdTiles) {
            const int nt = min(kIdTiles, T - sc);
            if (prod_or(false)) break;   // every producer is done with the previous ids
            const int64_t pbase = (c0 + sc) * kM;
            for (int i = tid; i < nt * kM; i += kProdThreads) {
                const int64_t pos = pbase + i;
                sid[i] = pos < total ? a.ids[pos] : -1;
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
                    const int kb = sg * kbs + kbl;
                    const uint32_t dst = smem_u32(Asm + (size_t)st * stage_bytes + (size_t)kbl * kKB);
                    for (int i = 0; i < 32 / rpi; ++i) {
                        const int r = warp + 4 * (i * rpi + rl);
                        const int32_t id = sid[tt * kM + r];
                        const unsigned char *src =
                            id >= 0 ? Xp + (int64_t)id * row_bytes + kb * kBK + cc * 16 : Xp;
                        cp_async16(dst + sw128_offset(r, cc), src, id >= 0 ? 16u : 0u);
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
        const int lq = warp & 3;                 // TMEM lane quarter of this warp
        const int row = lq * 32 + lane;          // row within the tile
        const float mulc = a.metric == 0 ? -2.0f : -1.0f;
        auto valid_at = [&](int t) { return t < T && (c0 + t) * kM + row < total; };
        auto id_at = [&](int t) -> int32_t { return valid_at(t) ? a.ids[(c0 + t) * kM + row] : 0; };
        auto xn_of = [&](int t, int32_t id) -> float {
            return (valid_at(t) && a.metric == 0) ? __ldg(a.xnorm + id) : 0.0f;
        };
        int32_t id_n = id_at(1);
        float xn_c = xn_of(0, id_at(0));
        for (int t = 0; t < T; ++t) {
            const int acc = t & 1, use = t >> 1;
            const int64_t pos = (c0 + t) * kM + row;
            const bool valid = pos < total;
            const float xn = xn_c;
            xn_c = xn_of(t + 1, id_n);
            id_n = id_at(t + 2);
            const bool okw = warp_wait(&accfull[acc], use & 1, abort_flag);
            if (epi_or(!okw)) {
                if (!okw && lane == 0) fail();
                break;
            }
            tc_fence_after();
            const uint32_t tbase = tmem_base + ((uint32_t)(lq * 32) << 16) + (uint32_t)(acc * 2 * NQ);
            constexpr int kChunks = (2 * NQ + 31) / 32;
            float key[NQ];
#pragma unroll
            for (int ch = 0; ch < kChunks; ++ch) {
                uint32_t v[32];
                tmem_ld32(tbase + ch * 32, v);
                tmem_ld_wait();
                // columns [0, NQ): q1.x1 + q1.x2; [NQ, 2 NQ): q2.x1
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int col = ch * 32 + i;
                    if (col < NQ) key[col] = __uint_as_float(v[i]);
                    else if (col < 2 * NQ) key[col - NQ] += __uint_as_float(v[i]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty[acc]);
            const int buf = t & 1;
#pragma unroll
            for (int j = 0; j < NQ; ++j) {
                float k = a.metric == 0 ? fmaxf(qn[j] + xn + mulc * key[j], 0.0f) : -key[j];
                uint32_t m = 0xffffffffu;
                if (valid && q0 + j < a.B) {
                    a.keys_out[(int64_t)(q0 + j) * a.keys_ld + pos] = k;
                    m = float_to_ordered(k);
                }
                m = __reduce_min_sync(0xffffffffu, m);
                if (lane == 0 && q0 + j < a.B) atomicMin(&cmin_s[buf][j], m);
            }
            epi_or(false);
            const int et = tid - (kProdThreads + 32);
            if (et < NQ) {
                if (q0 + et < a.B)
                    a.chunk_min[(int64_t)(q0 + et) * a.cmin_ld + c0 + t] = cmin_s[buf][et];
                cmin_s[buf][et] = 0xffffffffu;   // reused two tiles later, after a barrier
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

int pair_nq(int B) { return B <= 16 ? 16 : B <= 32 ? 32 : 64; }

// Stages that fit next to the B operand (3 or 2, or 4 of 32 KB).
int pair_stages(int ldp, int nq) {
    for (int ns : {4, 3, 2}) {
        if (ns == 4 && pair_kbs(ldp) != 2) continue;
        if (playout(ldp, nq, ns).total <= (size_t)227 * 1024) return ns;
    }
    return 0;
}

template <int NQ, int NS>
cudaError_t launch_t(const ScanArgs &a, const unsigned char *Xp, int ldp, int G, cudaStream_t s) {
    const size_t sm = playout(ldp, NQ, NS).total;
    cudaError_t e = cudaFuncSetAttribute(umma_pair_kernel<NQ, NS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int nqt = (a.B + NQ - 1) / NQ;
    return launch_dependent(umma_pair_kernel<NQ, NS>, dim3(nqt * G), dim3(kThreads), sm, s, a, Xp,
                            ldp);
}

template <int NQ>
cudaError_t launch_nq(const ScanArgs &a, const unsigned char *Xp, int ldp, int G, int ns,
                      cudaStream_t s) {
    switch (ns) {
        case 4: return launch_t<NQ, 4>(a, Xp, ldp, G, s);
        case 3: return launch_t<NQ, 3>(a, Xp, ldp, G, s);
        default: return launch_t<NQ, 2>(a, Xp, ldp, G, s);
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
    switch (nq) {
        case 16: return launch_nq<16>(a, xp, ldp, G, ns, s);
        case 32: return launch_nq<32>(a, xp, ldp, G, ns, s);
        default: return launch_nq<64>(a, xp, ldp, G, ns, s);
    }
}

}  // namespace vrs
