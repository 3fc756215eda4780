// k_gemv.cu -- fused FP32 scan for small query batches: the on-the-fly
// predicate strategy of Sec. 3.2 ("the relational filter is checked, and if
// the condition is satisfied, the vector comparison takes place") for the
// per-tuple scan strategies 1:N / N:1 of Sec. 3.1, as one kernel:
// predicate, gather of the qualifying rows, distance, per-CTA top-k'.
//
// Each CTA owns a contiguous range of the table and runs two roles:
//   warp 8 (producer): evaluates theta_R 128 rows at a time from 16-byte
//     attribute loads, and copies every qualifying row into the next free
//     slot of a shared-memory stage with one bulk copy (cp.async.bulk, TMA
//     engine) per row, completing on the stage's mbarrier; row slots are
//     padded by 64 bytes so the consumers' 16-byte reads are conflict-free.
//   warps 0-7 (consumers): four lanes per row, two rows per lane; queries
//     sit in shared memory in a lane-skewed layout; the dot products use
//     packed two-wide FP32 FMAs (fma.rn.f32x2, two queries per
//     instruction); then the first-pass key (L2: ||q||^2 - 2 q.x + ||x||^2,
//     IP: -q.x) goes through the same candidate buffers / radix-select cut
//     / global bound as the CUDA-core scan, and survivors are appended.
// Stages are released right after the arithmetic, so the producer refills
// while the consumers select.  Every wait is bounded (error word on
// timeout; the producer drains its copies before the CTA exits).
#include "topk_select.cuh"
#include "umma.cuh"
#include "vrs_internal.cuh"

namespace vrs {
namespace {

using namespace umma;

constexpr int kCons = 256;                 // consumer threads
constexpr int kThreads = kCons + 32;       // + producer warp
constexpr int kWarps = kCons / 32;
constexpr int kRPL = 2;                    // rows per lane
constexpr int kR = (kCons / 4) * kRPL;     // rows per stage: 128
constexpr int kNS = 2;                     // stages
constexpr int kPadBytes = 64;

struct GLayout {
    size_t q_off, qn_off, stage_off, ids_off, n_off, bar_off, cnt_off, tau_off, taul_off,
        hist_off, buf_off, total;
    int region;    // floats per query region (ld/4 * QB + 8)
    int slot;      // bytes per row slot
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline GLayout glayout(int QB, int ld, int cap) {
    GLayout L;
    L.region = ld / 4 * QB + 8;
    L.slot = ld * 4 + kPadBytes;
    size_t o = 0;
    L.q_off = o;
    o += al16((size_t)4 * L.region * 4);
    L.qn_off = o;
    o += al16(QB * 4);
    o = (o + 127) & ~size_t(127);
    L.stage_off = o;
    o += (size_t)kNS * kR * L.slot;
    L.ids_off = o;
    o += al16((size_t)kNS * kR * 4);
    L.n_off = o;
    o += 16;
    L.bar_off = o;
    o += al16(2 * kNS * 8 + 8);
    L.cnt_off = o;
    o += al16(QB * 4);
    L.tau_off = o;
    o += al16(QB * 8);
    L.taul_off = o;
    o += al16(QB * 8);
    L.hist_off = o;
    o += al16(kWarps * 256 * 4);
    L.buf_off = o;
    o += (size_t)QB * cap * 8;
    L.total = o;
    return L;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool bar_cons_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, 256, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ uint64_t pack2(float x) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void ffma2(uint64_t &acc, uint64_t a, uint64_t b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}

// Reduce acc over the 4 lanes of a row (see the CUDA-core scan for the
// ownership rule: for QB >= 4 each lane ends with one quarter of the queries).
template <int QB>
__device__ __forceinline__ void reduce4g(float (&acc)[kRPL][QB], int sub) {
    if constexpr (QB >= 4) {
        constexpr int H = QB / 2, Qr = QB / 4;
        const bool b0 = sub & 1, b1 = (sub >> 1) & 1;
#pragma unroll
        for (int r = 0; r < kRPL; ++r) {
#pragma unroll
            for (int j = 0; j < H; ++j) {
                float mine = b0 ? acc[r][j + H] : acc[r][j];
                float other = b0 ? acc[r][j] : acc[r][j + H];
                acc[r][j] = mine + __shfl_xor_sync(0xffffffffu, other, 1);
            }
#pragma unroll
            for (int j = 0; j < Qr; ++j) {
                float mine = b1 ? acc[r][j + Qr] : acc[r][j];
                float other = b1 ? acc[r][j] : acc[r][j + Qr];
                acc[r][j] = mine + __shfl_xor_sync(0xffffffffu, other, 2);
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < kRPL; ++r)
#pragma unroll
            for (int j = 0; j < QB; ++j) {
                acc[r][j] += __shfl_xor_sync(0xffffffffu, acc[r][j], 1);
                acc[r][j] += __shfl_xor_sync(0xffffffffu, acc[r][j], 2);
            }
    }
}

__device__ __forceinline__ bool in_rng(int32_t a, int32_t lo, int32_t hi) { return lo <= a && a < hi; }

template <int QB>
__global__ void __launch_bounds__(kThreads, 1)
gemv_fused_kernel(GemvArgs a, int cap) {
    extern __shared__ __align__(128) unsigned char sm[];
    const int ld = a.ld;
    const GLayout L = glayout(QB, ld, cap);
    float *Qs = reinterpret_cast<float *>(sm + L.q_off);
    float *qn = reinterpret_cast<float *>(sm + L.qn_off);
    unsigned char *stages = sm + L.stage_off;
    int32_t *sids = reinterpret_cast<int32_t *>(sm + L.ids_off);
    int32_t *sn = reinterpret_cast<int32_t *>(sm + L.n_off);
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + L.bar_off), *empty = full + kNS;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + kNS);
    int *cnt = reinterpret_cast<int *>(sm + L.cnt_off);
    uint64_t *tau = reinterpret_cast<uint64_t *>(sm + L.tau_off);
    uint64_t *tau_local = reinterpret_cast<uint64_t *>(sm + L.taul_off);
    int *hist = reinterpret_cast<int *>(sm + L.hist_off);
    uint64_t *buf = reinterpret_cast<uint64_t *>(sm + L.buf_off);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q0 = blockIdx.x * QB;
    const int G = gridDim.y, g = blockIdx.y;
    // row ranges on 128-row chunk boundaries (16-byte attribute loads)
    const int64_t n_chunks = (a.n + 127) / 128;
    const int64_t r0 = 128 * (n_chunks * g / G);
    const int64_t r1 = min(a.n, 128 * (n_chunks * (g + 1) / G));
    const int kp = a.kp;

    // queries -> lane-skewed layout: dim (16t + 4s + i) of query j lives in
    // region s at (4t + i) * QB + j
    for (int idx = tid; idx < QB * ld; idx += kThreads) {
        const int j = idx / ld, dd = idx - j * ld;
        const int t = dd >> 4, s = (dd >> 2) & 3, i = dd & 3;
        const float v = (q0 + j < a.B && dd < a.d) ? a.Q[(int64_t)(q0 + j) * a.ldq + dd] : 0.0f;
        Qs[s * L.region + (4 * t + i) * QB + j] = v;
    }
    for (int j = tid; j < QB; j += kThreads) {
        cnt[j] = 0;
        tau[j] = kEmpty;
        tau_local[j] = kEmpty;
        float s2 = 0.0f;
        if (q0 + j < a.B)
            for (int dd = 0; dd < a.d; ++dd) {
                const float v = a.Q[(int64_t)(q0 + j) * a.ldq + dd];
                s2 = fmaf(v, v, s2);
            }
        qn[j] = s2;
    }
    if (tid == 0) {
        for (int i = 0; i < kNS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kWarps);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    auto fail = [&]() {
        *abort_flag = 1;
        atomicExch(a.err, 1);
    };

    if (warp == kWarps) {
        // ---------------------------------------------------------- producer
        const uint32_t row_bytes = (uint32_t)ld * 4;
        int it = 0, fill = 0;
        bool ok = true;
        int st = 0;
        int last_use[kNS];
        for (int i = 0; i < kNS; ++i) last_use[i] = -1;
        auto open_stage = [&]() -> bool {
            st = it % kNS;
            return mbar_wait(&empty[st], ((it / kNS) & 1) ^ 1, abort_flag);
        };
        auto close_stage = [&](int n_rows) {
            if (lane == 0) sn[st] = n_rows;
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[st]);
            last_use[st] = it;
            ++it;
        };
        ok = __all_sync(0xffffffffu, open_stage());
        for (int64_t c0 = r0; c0 < r1 && ok; c0 += 128) {
            const int64_t rb = c0 + lane * 4;
            uint32_t nib = 0;
            if (rb + 3 < r1) {
                uint32_t m = 0xFu;
                for (int t = 0; t < a.pred.n_terms; ++t) {
                    const int4 v = *reinterpret_cast<const int4 *>(a.attrs.col[a.pred.col[t]] + rb);
                    const int32_t lo = a.pred.lo[t], hi = a.pred.hi[t];
                    m &= (uint32_t)in_rng(v.x, lo, hi) | ((uint32_t)in_rng(v.y, lo, hi) << 1) |
                         ((uint32_t)in_rng(v.z, lo, hi) << 2) | ((uint32_t)in_rng(v.w, lo, hi) << 3);
                }
                nib = m;
            } else {
                for (int i = 0; i < 4; ++i) {
                    const int64_t r = rb + i;
                    if (r >= r1) break;
                    bool sel = true;
                    for (int t = 0; t < a.pred.n_terms; ++t)
                        sel = sel && in_rng(a.attrs.col[a.pred.col[t]][r], a.pred.lo[t], a.pred.hi[t]);
                    nib |= (uint32_t)sel << i;
                }
            }
            const int cl = __popc(nib);
            int incl = cl;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            if (a.count_out && blockIdx.x == 0 && lane == 0 && total)
                atomicAdd(reinterpret_cast<unsigned long long *>(a.count_out),
                          (unsigned long long)total);
            if (total == 0) continue;
            const int excl = incl - cl;
            const int n1 = min(total, kR - fill);
            // part 1: into the current stage
            if (lane == 0) mbar_expect_tx(&full[st], (uint32_t)n1 * row_bytes);
            __syncwarp();
            {
                int o = excl;
                for (int i = 0; i < 4; ++i) {
                    if (!((nib >> i) & 1)) continue;
                    if (o < n1) {
                        const int slot = fill + o;
                        const int32_t row = (int32_t)(rb + i);
                        sids[st * kR + slot] = row;
                        bulk_g2s(smem_u32(stages + ((size_t)st * kR + slot) * L.slot),
                                 a.X + (int64_t)row * ld, row_bytes, &full[st]);
                    }
                    ++o;
                }
            }
            fill += n1;
            if (fill == kR) {
                close_stage(kR);
                fill = 0;
                ok = __all_sync(0xffffffffu, open_stage());
                if (!ok) break;
            }
            if (total > n1) {
                // part 2: the rest into the fresh stage
                const int n2 = total - n1;
                if (lane == 0) mbar_expect_tx(&full[st], (uint32_t)n2 * row_bytes);
                __syncwarp();
                int o = excl;
                for (int i = 0; i < 4; ++i) {
                    if (!((nib >> i) & 1)) continue;
                    if (o >= n1) {
                        const int slot = o - n1;
                        const int32_t row = (int32_t)(rb + i);
                        sids[st * kR + slot] = row;
                        bulk_g2s(smem_u32(stages + ((size_t)st * kR + slot) * L.slot),
                                 a.X + (int64_t)row * ld, row_bytes, &full[st]);
                    }
                    ++o;
                }
                fill = n2;
            }
        }
        if (ok) {
            if (fill > 0) {
                close_stage(fill);
                fill = 0;
                ok = __all_sync(0xffffffffu, open_stage());
            }
            if (ok) close_stage(-1);   // end-of-range sentinel
        }
        if (!ok) {
            if (lane == 0) fail();
            // copies may still be in flight into the open stage and into
            // closed stages the consumers never took: close the open one and
            // wait (bounded) for every stage's last phase before exiting
            volatile int never = 0;
            if (fill > 0) {
                if (lane == 0) mbar_arrive(&full[st]);
                last_use[st] = it;
            }
            if (lane == 0)
                for (int i = 0; i < kNS; ++i)
                    if (last_use[i] >= 0) mbar_wait(&full[i], (last_use[i] / kNS) & 1, &never);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------- consumers
        const int sub = lane & 3, slotbase = warp * 8 + (lane >> 2);
        const float *Qr = Qs + sub * L.region;
        int it = 0;
        bool ok = true;
        while (true) {
            const int st = it % kNS;
            ok = __all_sync(0xffffffffu, mbar_wait(&full[st], (it / kNS) & 1, abort_flag));
            if (bar_cons_or(!ok)) {
                if (tid == 0) fail();
                break;
            }
            const int n_rows = sn[st];
            if (n_rows < 0) break;
            const unsigned char *sb = stages + (size_t)st * kR * L.slot;
            float acc[kRPL][QB];
            int32_t row[kRPL];
            bool valid[kRPL];
#pragma unroll
            for (int r = 0; r < kRPL; ++r) {
                const int slot = slotbase + r * (kR / kRPL);
                valid[r] = slot < n_rows;
                row[r] = valid[r] ? sids[st * kR + slot] : 0;
            }
            if constexpr (QB >= 2) {
                uint64_t acc2[kRPL][QB / 2];
#pragma unroll
                for (int r = 0; r < kRPL; ++r)
#pragma unroll
                    for (int j = 0; j < QB / 2; ++j) acc2[r][j] = 0ull;
                for (int t = 0; t < ld / 16; ++t) {
                    float4 x[kRPL];
#pragma unroll
                    for (int r = 0; r < kRPL; ++r) {
                        const int slot = slotbase + r * (kR / kRPL);
                        x[r] = *reinterpret_cast<const float4 *>(sb + (size_t)slot * L.slot +
                                                                 (size_t)(t * 16 + sub * 4) * 4);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const uint64_t *qp =
                            reinterpret_cast<const uint64_t *>(Qr + (4 * t + i) * QB);
                        uint64_t qv[QB / 2];
#pragma unroll
                        for (int j = 0; j < QB / 2; ++j) qv[j] = qp[j];
#pragma unroll
                        for (int r = 0; r < kRPL; ++r) {
                            const float xs = i == 0 ? x[r].x : i == 1 ? x[r].y : i == 2 ? x[r].z : x[r].w;
                            const uint64_t xx = pack2(xs);
#pragma unroll
                            for (int j = 0; j < QB / 2; ++j) ffma2(acc2[r][j], qv[j], xx);
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < kRPL; ++r)
#pragma unroll
                    for (int j = 0; j < QB / 2; ++j) {
                        acc[r][2 * j] = __uint_as_float((uint32_t)(acc2[r][j] & 0xffffffffu));
                        acc[r][2 * j + 1] = __uint_as_float((uint32_t)(acc2[r][j] >> 32));
                    }
            } else {
#pragma unroll
                for (int r = 0; r < kRPL; ++r) acc[r][0] = 0.0f;
                for (int t = 0; t < ld / 16; ++t) {
#pragma unroll
                    for (int r = 0; r < kRPL; ++r) {
                        const int slot = slotbase + r * (kR / kRPL);
                        const float4 x = *reinterpret_cast<const float4 *>(
                            sb + (size_t)slot * L.slot + (size_t)(t * 16 + sub * 4) * 4);
                        acc[r][0] = fmaf(Qr[4 * t + 0], x.x, acc[r][0]);
                        acc[r][0] = fmaf(Qr[4 * t + 1], x.y, acc[r][0]);
                        acc[r][0] = fmaf(Qr[4 * t + 2], x.z, acc[r][0]);
                        acc[r][0] = fmaf(Qr[4 * t + 3], x.w, acc[r][0]);
                    }
                }
            }
            // the stage's rows are no longer needed
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
            reduce4g<QB>(acc, sub);

            constexpr int OWN = QB >= 4 ? QB / 4 : QB;
            const int jbase = QB >= 4 ? ((sub & 1) * 2 + (sub >> 1)) * (QB / 4) : 0;
            const bool active = QB >= 4 || sub == 0;
#pragma unroll
            for (int r = 0; r < kRPL; ++r) {
                const float xn = (a.metric == 0 && valid[r]) ? __ldg(a.xnorm + row[r]) : 0.0f;
#pragma unroll
                for (int jj = 0; jj < OWN; ++jj) {
                    const int j = jbase + jj;
                    bool hit = false;
                    uint64_t c = 0;
                    if (valid[r] && active && q0 + j < a.B) {
                        const float dot = acc[r][jj];
                        const float key = a.metric == 0 ? fmaxf(qn[j] + xn - 2.0f * dot, 0.0f) : -dot;
                        c = make_cand(key, row[r]);
                        hit = c < tau[j];
                    }
                    if (__any_sync(0xffffffffu, hit)) {
                        const unsigned grp = __match_any_sync(0xffffffffu, hit ? j : -1);
                        const int leader = __ffs(grp) - 1;
                        int p = 0;
                        if (hit && lane == leader) p = atomicAdd(&cnt[j], __popc(grp));
                        p = __shfl_sync(0xffffffffu, p, leader);
                        if (hit) buf[(size_t)j * cap + p + __popc(grp & ((1u << lane) - 1u))] = c;
                    }
                }
            }
            bar_cons_or(false);
            for (int j = warp; j < QB; j += kWarps) {
                if (q0 + j >= a.B) continue;
                const int c = cnt[j];
                if (c > cap - kR || (c >= kp && tau_local[j] == kEmpty)) {
                    uint64_t *b = buf + (size_t)j * cap;
                    SelectResult sr = warp_select(b, c, kp, hist + warp * 256);
                    uint64_t mx;
                    const int kept = warp_pack(b, c, sr, &mx);
                    if (lane == 0) {
                        cnt[j] = kept;
                        tau_local[j] = mx;
                        atomicMin(reinterpret_cast<unsigned long long *>(a.tau_g + q0 + j),
                                  (unsigned long long)mx);
                    }
                }
                if (lane == 0) {
                    const uint64_t gg = *reinterpret_cast<volatile uint64_t *>(a.tau_g + q0 + j);
                    const uint64_t tl = tau_local[j];
                    tau[j] = gg < tl ? gg : tl;
                }
            }
            bar_cons_or(false);
            ++it;
        }
        // final cut to k' and append the survivors under the global bound
        if (ok) {
            for (int j = warp; j < QB; j += kWarps) {
                if (q0 + j >= a.B) continue;
                uint64_t *b = buf + (size_t)j * cap;
                int c = cnt[j];
                if (c > kp) {
                    SelectResult sr = warp_select(b, c, kp, hist + warp * 256);
                    uint64_t mx;
                    c = warp_pack(b, c, sr, &mx);
                    if (lane == 0)
                        atomicMin(reinterpret_cast<unsigned long long *>(a.tau_g + q0 + j),
                                  (unsigned long long)mx);
                } else if (c == kp) {
                    uint64_t mx = 0;
                    for (int i = lane; i < c; i += 32) mx = b[i] > mx ? b[i] : mx;
#pragma unroll
                    for (int o = 16; o; o >>= 1) {
                        const uint64_t y = __shfl_xor_sync(0xffffffffu, mx, o);
                        mx = y > mx ? y : mx;
                    }
                    if (lane == 0)
                        atomicMin(reinterpret_cast<unsigned long long *>(a.tau_g + q0 + j),
                                  (unsigned long long)mx);
                }
                __syncwarp();
                const uint64_t gb = *reinterpret_cast<volatile uint64_t *>(a.tau_g + q0 + j);
                uint64_t *o = a.out + (int64_t)(q0 + j) * a.out_cap;
                for (int base = 0; base < c; base += 32) {
                    const int i = base + lane;
                    const bool keep = i < c && b[i] <= gb;
                    const unsigned bal = __ballot_sync(0xffffffffu, keep);
                    int pos = 0;
                    if (lane == 0 && bal) pos = atomicAdd(a.out_cnt + q0 + j, __popc(bal));
                    pos = __shfl_sync(0xffffffffu, pos, 0);
                    if (keep) {   // past the list's end: nothing written, error word set
                        const int slot = pos + __popc(bal & ((1u << lane) - 1u));
                        if (slot < a.out_cap) o[slot] = b[i];
                        else atomicExch(a.err, 2);
                    }
                }
            }
        }
    }
    __syncthreads();
}

template <int QB>
cudaError_t launch_g(const GemvArgs &a, int G, cudaStream_t s) {
    const int cap = a.kp + 2 * kR;
    const GLayout L = glayout(QB, a.ld, cap);
    cudaError_t e = cudaFuncSetAttribute(gemv_fused_kernel<QB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    dim3 grid((a.B + QB - 1) / QB, G);
    gemv_fused_kernel<QB><<<grid, kThreads, L.total, s>>>(a, cap);
    return cudaGetLastError();
}

}  // namespace

// Shared memory of the fused scan for a query group of QB (host check).
size_t gemv_fused_smem(int QB, int ld, int kp) { return glayout(QB, ld, kp + 2 * kR).total; }

int gemv_fused_query_block(int B) {
    if (B <= 1) return 1;
    if (B <= 2) return 2;
    if (B <= 4) return 4;
    if (B <= 8) return 8;
    return 16;
}

cudaError_t launch_gemv_fused(const GemvArgs &a, int G, cudaStream_t s) {
    const int QB = gemv_fused_query_block(a.B);
    if (gemv_fused_smem(QB, a.ld, a.kp) > 227 * 1024 || a.err == nullptr) return cudaErrorInvalidValue;
    switch (QB) {
        case 1: return launch_g<1>(a, G, s);
        case 2: return launch_g<2>(a, G, s);
        case 4: return launch_g<4>(a, G, s);
        case 8: return launch_g<8>(a, G, s);
        default: return launch_g<16>(a, G, s);
    }
}

}  // namespace vrs
