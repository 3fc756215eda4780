// k_umma_rows.cu -- the dense-key distance pass for small query batches on
// the tensor cores: 128 selected rows per tile are the MMA's M dimension and
// the (few) queries its N dimension, so the tensor core does the arithmetic
// that would otherwise bound a CUDA-core scan at 16+ queries, and the kernel
// is left with the gather of the rows.
//
// Arithmetic: FP32 rows and queries are split exactly into a TF32 high part
// and a remainder, x = xh + xl with xh = x with its low 13 mantissa bits
// cleared, and q . x ~= qh . xh + ql . xh + qh . xl (the "3xTF32" scheme:
// each product pair is formed by the tensor core from TF32 operands and
// accumulated in FP32; the dropped ql . xl term and the TF32 reading of the
// remainders leave a relative error of a few 2^-21 per product).  The B
// operand holds [qh ; ql] as 2 NQ rows, so per K step one MMA of N = 2 NQ
// gives qh . xh and ql . xh and a second MMA of N = NQ adds qh . xl into the
// first NQ columns.  Keys: L2 max(||q||^2 + ||x||^2 - 2 q.x, 0), IP -q.x; the
// exact FP32 re-rank of the k' best follows in the merge.
//
// Warp roles (416 threads):
//   warps 0-7   split warps: the row ids of up to 64 tiles go to shared
//               memory first; then each thread loads 64 bytes of a row per
//               K block (16-byte global loads, issued PF K blocks ahead), writes the
//               high and low parts into the 128-byte-swizzled K-major A
//               stages, fences the async proxy and hands the stage over;
//   warp 8      allocates TMEM and, from one lane, issues tcgen05.mma
//               (kind::tf32, M = 128) and the commits that free stages and
//               publish accumulators (double-buffered);
//   warps 9-12  epilogue: tcgen05.ld of a row's 2 NQ accumulator columns
//               (TMEM lane = row), the keys written to the dense key matrix,
//               and the per-query minimum over the tile (= one 128-position
//               chunk) written to the chunk-minimum array.
// Every mbarrier wait is bounded; on timeout the kernel records an error in
// *err, lets the MMAs drain, frees its TMEM and returns.
#include <algorithm>

#include "umma.cuh"
#include "vrs_internal.cuh"

namespace vrs {
namespace {

using namespace umma;

constexpr int kM = 128;                  // rows per tile (TMEM lanes)
constexpr int kBK = 128;                 // bytes of K per stage (one swizzle atom)
constexpr int kSplitWarps = 8;
constexpr int kSplitThreads = kSplitWarps * 32;
constexpr int kEpiThreads = 128;
constexpr int kThreads = kSplitThreads + 32 + kEpiThreads;   // 416
constexpr int kPF = 6;                   // K blocks loaded ahead per split thread
constexpr int kAHalf = kM * kBK;         // 16 KB: one operand half of a stage
constexpr int kIdTiles = 64;             // tiles whose row ids are staged at a time
constexpr int kBuilders = kThreads - kSplitThreads;   // MMA + epilogue threads: 160

struct RLayout {
    int nkb, ns;
    size_t b_off, a_off, bar_off, qn_off, total;
};

__host__ __device__ inline size_t ral(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline RLayout rlayout(int row_bytes, int nq, int ns) {
    RLayout L;
    L.nkb = (row_bytes + kBK - 1) / kBK;
    L.ns = ns;
    size_t o = 0;
    L.b_off = o;                                  // [nkb][2 nq rows x 128 B]
    o += (size_t)L.nkb * 2 * nq * kBK;
    o = ral(o, 1024);
    L.a_off = o;                                  // [ns][hi 16 KB | lo 16 KB]
    o += (size_t)ns * 2 * kAHalf;
    L.bar_off = o;                                // full, empty, accfull x2, accempty x2, done
    o += ral((size_t)(2 * ns + 5) * 8 + 16, 16);
    L.qn_off = o;
    o += ral((size_t)nq * 4, 16);
    L.total = o + 1024;                           // slack for 1024-byte alignment
    return L;
}

// TMEM columns: two accumulators of 2 NQ columns, rounded to a power of two >= 32.
__host__ __device__ constexpr uint32_t tmem_cols(int nq) {
    return 4 * nq <= 32 ? 32u : 4 * nq <= 64 ? 64u : 4 * nq <= 128 ? 128u : 256u;
}

// The TF32 high part of x: sign, exponent and the top 10 mantissa bits.
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xffffe000u); }

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

__device__ __forceinline__ void split_sync() {
    asm volatile("bar.sync 2, %0;" ::"n"(kSplitThreads) : "memory");
}
__device__ __forceinline__ bool split_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 2, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kSplitThreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void builders_sync() {
    asm volatile("bar.sync 3, %0;" ::"n"(kBuilders) : "memory");
}

__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
    return __all_sync(0xffffffffu, mbar_wait(bar, parity, abort));
}

template <int NQ>
__global__ void __launch_bounds__(kThreads, 1)
umma_rows_kernel(ScanArgs a, int ns) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw_u32 = smem_u32(smem_raw);
    unsigned char *sm = smem_raw + (((raw_u32 + 1023u) & ~1023u) - raw_u32);
    const int row_bytes = a.ld * 4;
    const RLayout L = rlayout(row_bytes, NQ, ns);
    const int nkb = L.nkb;
    unsigned char *Bsm = sm + L.b_off;
    unsigned char *Asm = sm + L.a_off;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L.bar_off);
    uint64_t *full = bars, *empty = bars + ns, *accfull = bars + 2 * ns,
             *accempty = bars + 2 * ns + 2, *done = bars + 2 * ns + 4;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * ns + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    float *qn = reinterpret_cast<float *>(sm + L.qn_off);
    __shared__ uint32_t cmin_s[2][NQ];
    __shared__ __align__(16) int32_t sid[kIdTiles * kM];   // row ids of a super-chunk
    constexpr uint32_t kCols = tmem_cols(NQ);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nqt = (a.B + NQ - 1) / NQ;
    const int qt = blockIdx.x % nqt, g = blockIdx.x / nqt, G = gridDim.x / nqt;
    const int q0 = qt * NQ;
    // launched as a programmatic dependent of the filter kernel: the set-up
    // below (barriers, TMEM, the query operand) overlaps its tail, and the
    // selected-row count and ids are read only after griddepcontrol.wait
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    if (tid == 0) {
        for (int i = 0; i < ns; ++i) {
            mbar_init(&full[i], kSplitWarps);
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
    if (warp == kSplitWarps) {
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

    if (warp >= kSplitWarps) {
        // MMA and epilogue warps build the B operand, [qh ; ql] of this CTA's
        // queries (zero past B and past ld), 128-byte-swizzled K-major, and
        // ||q||^2 in plain float32, while the split warps start their loads
        const int bt = tid - kSplitThreads;
        for (int idx = bt; idx < nkb * 2 * NQ * 8; idx += kBuilders) {
            const int c = idx & 7, r = (idx >> 3) % (2 * NQ), kb = (idx >> 3) / (2 * NQ);
            const int j = r % NQ, off = kb * kBK + c * 16;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q0 + j < a.B && off < row_bytes)
                v = *reinterpret_cast<const float4 *>(a.Q + (int64_t)(q0 + j) * a.ld + off / 4);
            const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
            const float4 o = r < NQ ? h : make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
            *reinterpret_cast<float4 *>(Bsm + (size_t)kb * 2 * NQ * kBK + sw128_offset(r, c)) = o;
        }
        for (int j = warp - kSplitWarps; j < NQ; j += kBuilders / 32) {
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
    if (a.count_copy && blockIdx.x == 0 && tid == 0) *a.count_copy = total;
    const int64_t nch = (total + kM - 1) / kM;
    const int64_t c0 = nch * g / G, c1 = nch * (g + 1) / G;
    const int T = (int)(c1 - c0);

    if (warp < kSplitWarps) {
        // ------------------------------------------------------------ split
        // thread: row r of the tile, 16-byte units u0..u0+3 of each K block.
        // The row ids of up to kIdTiles tiles are staged in shared memory
        // first, so that the row loads (issued kPF steps ahead) never wait
        // on an id load.
        const int r = tid >> 1, u0 = (tid & 1) * 4;
        const unsigned char *X = reinterpret_cast<const unsigned char *>(a.X);
        auto load = [&](int s, uint4 (&v)[4]) {   // step s of the current super-chunk
            const int32_t id = sid[(s / nkb) * kM + r];
            const int kb = s % nkb;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int off = kb * kBK + (u0 + u) * 16;
                v[u] = (id >= 0 && off < row_bytes)
                           ? __ldg(reinterpret_cast<const uint4 *>(X + (int64_t)id * row_bytes + off))
                           : make_uint4(0, 0, 0, 0);
            }
        };
        bool ok = true;
        int sg = 0;   // global step (stage ring position)
        for (int sc = 0; sc < T && ok; sc += kIdTiles) {
            const int nt = min(kIdTiles, T - sc);
            split_sync();   // every split thread is done with the previous ids
            const int64_t pbase = (c0 + sc) * kM;
            for (int i = tid * 4; i < nt * kM; i += kSplitThreads * 4) {
                const int64_t pos = pbase + i;
                int4 v;
                if (pos + 3 < total) {
                    v = __ldg(reinterpret_cast<const int4 *>(a.ids + pos));
                } else {
                    v.x = pos < total ? a.ids[pos] : -1;
                    v.y = pos + 1 < total ? a.ids[pos + 1] : -1;
                    v.z = pos + 2 < total ? a.ids[pos + 2] : -1;
                    v.w = -1;
                }
                *reinterpret_cast<int4 *>(sid + i) = v;
            }
            split_sync();
            const int steps = nt * nkb;
            uint4 buf[kPF][4];
#pragma unroll
            for (int p = 0; p < kPF; ++p)
                if (p < steps) load(p, buf[p]);
            for (int s0 = 0; s0 < steps && ok; s0 += kPF) {
#pragma unroll
                for (int p = 0; p < kPF; ++p) {
                    const int s = s0 + p;
                    if (s >= steps) break;
                    const int st = sg % ns;
                    if (!warp_wait(&empty[st], ((sg / ns) & 1) ^ 1, abort_flag)) {
                        if (lane == 0) fail();
                        ok = false;
                        break;
                    }
                    unsigned char *hi = Asm + (size_t)st * 2 * kAHalf, *lo = hi + kAHalf;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 x = *reinterpret_cast<const float4 *>(&buf[p][u]);
                        const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
                        const float4 l = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
                        const uint32_t o = sw128_offset(r, u0 + u);
                        *reinterpret_cast<float4 *>(hi + o) = h;
                        *reinterpret_cast<float4 *>(lo + o) = l;
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&full[st]);
                    ++sg;
                    if (s + kPF < steps) load(s + kPF, buf[p]);
                }
            }
            // stop together (the next super-chunk's barrier needs everyone)
            ok = !split_or(!ok);
        }
    } else if (warp == kSplitWarps) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t id_full = idesc(2, kM, 2 * NQ), id_half = idesc(2, kM, NQ);
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
                for (int kb = 0; kb < nkb; ++kb, ++s) {
                    const int st = s % ns;
                    if (!mbar_wait(&full[st], (s / ns) & 1, abort_flag)) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t ahi = smem_u32(Asm + (size_t)st * 2 * kAHalf), alo = ahi + kAHalf;
                    const uint32_t bk = bbase + (uint32_t)(kb * 2 * NQ * kBK);
#pragma unroll
                    for (int kk = 0; kk < kBK / 32; ++kk) {
                        mma_tf32(d, desc_sw128(ahi + kk * 32), desc_sw128(bk + kk * 32), id_full,
                                 (kb | kk) != 0 ? 1u : 0u);
                        mma_tf32(d, desc_sw128(alo + kk * 32), desc_sw128(bk + kk * 32), id_half, 1u);
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
        // row ids two tiles ahead and norms one tile ahead, so the key of a
        // tile never waits on a dependent pair of loads
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
                // columns [0, NQ): qh.xh + qh.xl; [NQ, 2 NQ): ql.xh
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
            const int et = tid - (kSplitThreads + 32);
            if (et < NQ) {
                if (q0 + et < a.B)
                    a.chunk_min[(int64_t)(q0 + et) * a.cmin_ld + c0 + t] = cmin_s[buf][et];
                cmin_s[buf][et] = 0xffffffffu;   // reused two tiles later, after a barrier
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == kSplitWarps) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kCols);
    }
}

template <int NQ>
cudaError_t launch_nq(const ScanArgs &a, int G, int ns, cudaStream_t s) {
    const size_t sm = rlayout(a.ld * 4, NQ, ns).total;
    cudaError_t e = cudaFuncSetAttribute(umma_rows_kernel<NQ>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int nqt = (a.B + NQ - 1) / NQ;
    return launch_dependent(umma_rows_kernel<NQ>, dim3(nqt * G), dim3(kThreads), sm, s, a, ns);
}

int rows_nq(int B) { return B <= 16 ? 16 : B <= 32 ? 32 : 64; }

int rows_stages(int ld, int nq) {
    for (int ns = 4; ns >= 2; --ns)
        if (rlayout(ld * 4, nq, ns).total + kIdTiles * kM * 4 <= (size_t)220 * 1024) return ns;
    return 0;
}

}  // namespace

bool umma_rows_fits(int B, int ld) { return rows_stages(ld, rows_nq(B)) > 0; }

int umma_rows_grid(int B, int n_sm) {
    const int nqt = (B + rows_nq(B) - 1) / rows_nq(B);
    return std::max(1, n_sm / nqt);
}

cudaError_t launch_umma_rows(const ScanArgs &a, int G, cudaStream_t s) {
    const int nq = rows_nq(a.B);
    const int ns = rows_stages(a.ld, nq);
    if (ns == 0 || a.x_bf16 || a.keys_out == nullptr || a.ids == nullptr ||
        a.count_dev == nullptr || a.chunk_min == nullptr || a.err == nullptr || a.ld % 16)
        return cudaErrorInvalidValue;
    switch (nq) {
        case 16: return launch_nq<16>(a, G, ns, s);
        case 32: return launch_nq<32>(a, G, ns, s);
        default: return launch_nq<64>(a, G, ns, s);
    }
}

}  // namespace vrs
