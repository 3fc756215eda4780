// k_scan_simt.cu -- FP32 distance pass on CUDA cores with a fused per-CTA
// top-k' (the per-tuple scan strategies 1:N and N:1 of Sec. 3.1, with the
// relational predicate applied before the distance, Sec. 3.2).
//
// Work split.  Grid = (query groups of QB queries) x (G row partitions).
// blockIdx.x runs over query groups so that the CTAs resident at one time
// share a row partition and re-read it from L2, not HBM.  Inside a CTA,
// four lanes cooperate on one row (each loads 16 contiguous bytes per step,
// so a warp reads 8 rows x 64 B per instruction, whole 32-byte sectors), and
// every lane carries RPL = 2 rows so that each query value loaded from
// shared memory feeds two FMAs.  The queries of the group live in shared
// memory for the whole kernel.
//
// Distance (L2): ||q||^2 - 2 q.x + ||x||^2 with the row norms computed at
// load time, clamped at 0; (IP): key = -q.x.  These first-pass keys only
// choose candidates: the k' best per query are re-ranked exactly later.
//
// Top-k'.  Each query has a candidate buffer in shared memory and a
// threshold tau (the worst composite currently kept).  A lane appends a
// (key, id) composite when it beats tau.  Between row batches, a buffer that
// could overflow on the next batch is cut back to exactly its k' best by a
// warp radix select, and tau becomes the k'-th best.  At the end each CTA
// writes its (unsorted) k' best per query, padded with kEmpty.
#include "topk_select.cuh"
#include "umma.cuh"
#include "vrs_internal.cuh"

namespace vrs {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kLanesPerRow = 4;
constexpr int kRPL = 2;
constexpr int kSlots = kThreads / kLanesPerRow;   // 64 row slots
constexpr int kRPI = kSlots * kRPL;               // rows per iteration: 128
// Row steps (16 floats each) loaded ahead per lane: 8 for small query
// groups, 4 for 16+ queries so that two CTAs fit an SM's register file.
template <int QB> __host__ __device__ constexpr int chunk_of() { return 4; }
template <int QB> __host__ __device__ constexpr int min_ctas_of() { return QB >= 32 ? 1 : (QB >= 8 ? 2 : 3); }

struct Smem {
    float *Q;        // [QB x ld]
    float *qn;       // [QB]
    int *cnt;        // [QB]
    uint64_t *tau;   // [QB] insertion bound: min(local k'-th best, global bound)
    uint64_t *tau_local; // [QB] this CTA's k'-th best (kEmpty until k' seen)
    int *hist;       // [kWarps x 256]
    uint64_t *buf;   // [QB x cap]
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// floats per lane-quarter region of the skewed query layout (QB >= 2)
// Elements per 16-byte lane load (4 float32 or 8 bf16) and the row steps
// of 64 bytes (four lanes x 16 bytes) covering ld elements.
__host__ __device__ constexpr int vec_of(bool bf) { return bf ? 8 : 4; }
__host__ __device__ inline int steps_of(int ld, bool bf) { return (ld * (bf ? 2 : 4) + 63) / 64; }

// floats per lane-quarter region of the skewed query layout (QB >= 2)
__host__ __device__ inline int qregion(int QB, int ld, bool bf) {
    return steps_of(ld, bf) * vec_of(bf) * QB + 8;
}

__host__ __device__ inline size_t qbytes(int QB, int ld, bool bf) {
    return QB >= 2 ? (size_t)4 * qregion(QB, ld, bf) * 4
                   : (size_t)steps_of(ld, bf) * 4 * vec_of(bf) * 4;
}

__host__ __device__ inline size_t smem_bytes(int QB, int ld, int cap, bool bf) {
    return align16(qbytes(QB, ld, bf)) + align16(QB * 4) + align16(QB * 4) + 2 * align16(QB * 8) +
           align16(kWarps * 256 * 4) + (size_t)QB * cap * 8;
}

__device__ inline Smem carve(unsigned char *p, int QB, int ld, int cap, bool bf) {
    Smem s;
    s.Q = reinterpret_cast<float *>(p);
    p += align16(qbytes(QB, ld, bf));
    s.qn = reinterpret_cast<float *>(p);
    p += align16(QB * 4);
    s.cnt = reinterpret_cast<int *>(p);
    p += align16(QB * 4);
    s.tau = reinterpret_cast<uint64_t *>(p);
    p += align16(QB * 8);
    s.tau_local = reinterpret_cast<uint64_t *>(p);
    p += align16(QB * 8);
    s.hist = reinterpret_cast<int *>(p);
    p += align16(kWarps * 256 * 4);
    s.buf = reinterpret_cast<uint64_t *>(p);
    return s;
}

__device__ __forceinline__ uint64_t pack2(float x) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(x));
    return r;
}
// acc.{x,y} += a.{x,y} * b.{x,y} (packed two-wide FP32 FMA)
__device__ __forceinline__ void ffma2(uint64_t &acc, uint64_t a, uint64_t b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}

// Reduce acc[r][j] over the 4 lanes of a row group.  Afterwards lane `sub`
// holds the full sums of queries j in its quarter: for QB >= 4, quarter q of
// [0, QB) is owned by the lane with sub == q (bit0 picks the half, bit1 the
// quarter inside it).  For QB < 4 every lane holds every sum.
template <int QB>
__device__ __forceinline__ void reduce4(float (&acc)[kRPL][QB], int sub) {
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

// Element i (0 <= i < VEC) of a lane's 16-byte load as float32.
template <bool BF>
__device__ __forceinline__ float elem(const uint4 &v, int i) {
    if constexpr (!BF) {
        return __uint_as_float(i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w);
    } else {
        const uint32_t w = (i >> 1) == 0 ? v.x : (i >> 1) == 1 ? v.y : (i >> 1) == 2 ? v.z : v.w;
        return __uint_as_float((i & 1) ? (w & 0xffff0000u) : (w << 16));
    }
}

// BF: rows stored as bf16 (widened to float32 for the FMAs) instead of float32.
template <int QB, bool BF>
__global__ void __launch_bounds__(kThreads, min_ctas_of<QB>())
scan_simt_kernel(ScanArgs a, int cap) {
    constexpr int kChunk = chunk_of<QB>();
    constexpr int VEC = vec_of(BF);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem S = carve(smem_raw, QB, a.ld, cap, BF);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sub = lane & 3, slot = warp * 8 + (lane >> 2);
    const int q0 = blockIdx.x * QB;
    const int G = gridDim.y, g = blockIdx.y;
    const int ld = a.ld;

    // queries of this group -> shared memory (zero rows past B and dims
    // past ld).  For QB >= 2 the layout is query-pair interleaved and skewed
    // per lane quarter: dim (4 VEC t + VEC s + i) of query j at region s,
    // (VEC t + i) * QB + j, so the four lanes of a row read different banks.
    const int steps = steps_of(ld, BF);
    const int span = steps * 4 * VEC;   // dims covered by the steps (>= ld)
    const int qreg = qregion(QB, ld, BF);
    for (int i = tid; i < QB * span; i += kThreads) {
        const int j = i / span, dd = i - j * span;
        const float v = (q0 + j < a.B && dd < ld) ? a.Q[(int64_t)(q0 + j) * ld + dd] : 0.0f;
        if constexpr (QB >= 2) {
            const int t = dd / (4 * VEC), s4 = (dd / VEC) & 3, ii = dd % VEC;
            S.Q[s4 * qreg + (VEC * t + ii) * QB + j] = v;
        } else {
            S.Q[dd] = v;
        }
    }
    for (int j = tid; j < QB; j += kThreads) {
        S.cnt[j] = 0;
        S.tau[j] = kEmpty;
        S.tau_local[j] = kEmpty;
    }
    __syncthreads();
    // ||q||^2 (plain float32; the first pass only ranks candidates)
    for (int j = warp; j < QB; j += kWarps) {
        float s = 0.0f;
        if (q0 + j < a.B)
            for (int t = lane; t < ld; t += 32) {
                const float v = a.Q[(int64_t)(q0 + j) * ld + t];
                s = fmaf(v, v, s);
            }
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) S.qn[j] = s;
    }

    const int64_t total = a.ids ? *a.count_dev : a.n_rows;
    if (a.count_copy && blockIdx.x == 0 && threadIdx.x == 0) *a.count_copy = total;
    // dense-key mode: partitions start on 128-position chunks, so each
    // iteration covers exactly chunk base / 128 of the key row
    int64_t p0, p1;
    if (a.keys_out) {
        const int64_t nch = (total + kRPI - 1) / kRPI;
        p0 = nch * g / G * kRPI;
        p1 = min(total, nch * (g + 1) / G * kRPI);
    } else {
        p0 = total * g / G;
        p1 = total * (g + 1) / G;
    }
    __shared__ uint32_t cmin_s[2][QB];   // per-chunk minima, double-buffered
    for (int j = tid; j < 2 * QB; j += kThreads) cmin_s[j / QB][j % QB] = 0xffffffffu;
    const int kp = a.kp;
    __syncthreads();

    for (int64_t base = p0; base < p1; base += kRPI) {
        int32_t row[kRPL];
        bool valid[kRPL];
        int64_t posr[kRPL];
#pragma unroll
        for (int r = 0; r < kRPL; ++r) {
            int64_t pos = base + slot + r * kSlots;
            posr[r] = pos;
            valid[r] = pos < p1;
            row[r] = 0;
            if (valid[r]) {
                row[r] = a.ids ? a.ids[pos] : (int32_t)pos;
                if (!a.ids && a.bitmap) valid[r] = (a.bitmap[pos >> 5] >> (pos & 31)) & 1u;
            }
        }
        float acc[kRPL][QB];
#pragma unroll
        for (int r = 0; r < kRPL; ++r)
#pragma unroll
            for (int j = 0; j < QB; ++j) acc[r][j] = 0.0f;

        // row norms are fetched with the rows (one round trip, not two)
        float xnr[kRPL];
#pragma unroll
        for (int r = 0; r < kRPL; ++r)
            xnr[r] = (a.metric == 0 && valid[r]) ? __ldg(a.xnorm + row[r]) : 0.0f;
        const int row_bytes = ld * (BF ? 2 : 4);
        const uint4 *xr[kRPL];
#pragma unroll
        for (int r = 0; r < kRPL; ++r)
            xr[r] = reinterpret_cast<const uint4 *>(
                        reinterpret_cast<const unsigned char *>(a.X) + (int64_t)row[r] * row_bytes) + sub;
        // Issue every load of a chunk of kChunk steps before any FMA, so each
        // lane has kRPL * kChunk 16-byte loads in flight.
        auto load = [&](int r, int t) -> uint4 {
            return (valid[r] && t < steps && t * 64 + sub * 16 < row_bytes) ? __ldg(xr[r] + t * 4)
                                                                         : make_uint4(0, 0, 0, 0);
        };
        if constexpr (QB >= 2) {
            // packed two-query FMAs: (q_j, q_j+1) x (x, x)
            uint64_t acc2[kRPL][QB / 2];
#pragma unroll
            for (int r = 0; r < kRPL; ++r)
#pragma unroll
                for (int j = 0; j < QB / 2; ++j) acc2[r][j] = 0ull;
            const float *Qr = S.Q + sub * qreg;
            for (int t0 = 0; t0 < steps; t0 += kChunk) {
                uint4 x[kRPL][kChunk];
#pragma unroll
                for (int u = 0; u < kChunk; ++u)
#pragma unroll
                    for (int r = 0; r < kRPL; ++r) x[r][u] = load(r, t0 + u);
#pragma unroll
                for (int u = 0; u < kChunk; ++u) {
                    if (t0 + u >= steps) break;
#pragma unroll
                    for (int i = 0; i < VEC; ++i) {
                        const uint64_t *qp =
                            reinterpret_cast<const uint64_t *>(Qr + (VEC * (t0 + u) + i) * QB);
                        uint64_t qv[QB / 2];
#pragma unroll
                        for (int j = 0; j < QB / 2; ++j) qv[j] = qp[j];
#pragma unroll
                        for (int r = 0; r < kRPL; ++r) {
                            const uint64_t xx = pack2(elem<BF>(x[r][u], i));
#pragma unroll
                            for (int j = 0; j < QB / 2; ++j) ffma2(acc2[r][j], qv[j], xx);
                        }
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
            for (int t0 = 0; t0 < steps; t0 += kChunk) {
                uint4 x[kRPL][kChunk];
#pragma unroll
                for (int u = 0; u < kChunk; ++u)
#pragma unroll
                    for (int r = 0; r < kRPL; ++r) x[r][u] = load(r, t0 + u);
#pragma unroll
                for (int u = 0; u < kChunk; ++u) {
                    if (t0 + u >= steps) break;
                    const float *qd = S.Q + (t0 + u) * 4 * VEC + sub * VEC;
#pragma unroll
                    for (int i = 0; i < VEC; ++i)
#pragma unroll
                        for (int r = 0; r < kRPL; ++r)
                            acc[r][0] = fmaf(qd[i], elem<BF>(x[r][u], i), acc[r][0]);
                }
            }
        }
        reduce4<QB>(acc, sub);

        if (a.keys_out) {
            // dense-key mode: every first-pass key goes to the key matrix,
            // and the minimum of each query over the chunk to chunk_min
            constexpr int OWNK = QB >= 4 ? QB / 4 : QB;
            const int jb = QB >= 4 ? ((sub & 1) * 2 + (sub >> 1)) * (QB / 4) : 0;
            uint32_t mn[OWNK];
#pragma unroll
            for (int jj = 0; jj < OWNK; ++jj) mn[jj] = 0xffffffffu;
            if (QB >= 4 || sub == 0) {
#pragma unroll
                for (int r = 0; r < kRPL; ++r) {
                    if (posr[r] >= p1) continue;
                    const float xn = xnr[r];
#pragma unroll
                    for (int jj = 0; jj < OWNK; ++jj) {
                        const int j = jb + jj;
                        if (q0 + j >= a.B) continue;
                        const float dot = acc[r][jj];
                        float key = a.metric == 0 ? fmaxf(S.qn[j] + xn - 2.0f * dot, 0.0f) : -dot;
                        if (!valid[r]) key = __int_as_float(0x7f800000);
                        a.keys_out[(int64_t)(q0 + j) * a.keys_ld + posr[r]] = key;
                        mn[jj] = min(mn[jj], float_to_ordered(key));
                    }
                }
            }
            // lanes with the same quarter hold the same queries: reduce over
            // the warp's 8 row slots, then over the warps in shared memory
            const int buf = (int)(((base - p0) / kRPI) & 1);
#pragma unroll
            for (int jj = 0; jj < OWNK; ++jj) {
                mn[jj] = min(mn[jj], __shfl_xor_sync(0xffffffffu, mn[jj], 4));
                mn[jj] = min(mn[jj], __shfl_xor_sync(0xffffffffu, mn[jj], 8));
                mn[jj] = min(mn[jj], __shfl_xor_sync(0xffffffffu, mn[jj], 16));
                if (lane < 4 && (QB >= 4 || sub == 0) && q0 + jb + jj < a.B)
                    atomicMin(&cmin_s[buf][jb + jj], mn[jj]);
            }
            __syncthreads();
            if (tid < QB) {
                if (q0 + tid < a.B)
                    a.chunk_min[(int64_t)(q0 + tid) * a.cmin_ld + base / kRPI] = cmin_s[buf][tid];
                cmin_s[buf][tid] = 0xffffffffu;   // reused two iterations later, after a barrier
            }
            continue;
        }

        // candidate insertion: a lane appends (key, id) for each owned query
        // whose threshold it beats; lanes appending to the same query share
        // one shared-memory atomic.
        constexpr int OWN = QB >= 4 ? QB / 4 : QB;
        const int jbase = QB >= 4 ? ((sub & 1) * 2 + (sub >> 1)) * (QB / 4) : 0;
        const bool active = QB >= 4 || sub == 0;
#pragma unroll
        for (int r = 0; r < kRPL; ++r) {
            const float xn = xnr[r];
#pragma unroll
            for (int jj = 0; jj < OWN; ++jj) {
                const int j = jbase + jj;
                bool hit = false;
                uint64_t c = 0;
                if (valid[r] && active && q0 + j < a.B) {
                    float dot = acc[r][jj];
                    float key = a.metric == 0 ? fmaxf(S.qn[j] + xn - 2.0f * dot, 0.0f) : -dot;
                    c = make_cand(key, row[r]);
                    hit = c < S.tau[j];
                }
                if (__any_sync(0xffffffffu, hit)) {
                    const unsigned grp = __match_any_sync(0xffffffffu, hit ? j : -1);
                    const int leader = __ffs(grp) - 1;
                    int p = 0;
                    if (hit && lane == leader) p = atomicAdd(&S.cnt[j], __popc(grp));
                    p = __shfl_sync(0xffffffffu, p, leader);
                    if (hit) S.buf[(size_t)j * cap + p + __popc(grp & ((1u << lane) - 1u))] = c;
                }
            }
        }
        __syncthreads();
        // cut back buffers that could overflow on the next batch, and set the
        // first threshold as soon as a buffer holds k' candidates; publish
        // each CTA's k'-th best so every CTA filters against the best bound
        for (int j = warp; j < QB; j += kWarps) {
            if (q0 + j >= a.B) continue;
            int c = S.cnt[j];
            if (c > cap - kRPI || (c >= kp && S.tau_local[j] == kEmpty)) {
                uint64_t *b = S.buf + (size_t)j * cap;
                SelectResult sr = warp_select(b, c, kp, S.hist + warp * 256);
                uint64_t mx;
                int kept = warp_pack(b, c, sr, &mx);
                if (lane == 0) {
                    S.cnt[j] = kept;
                    S.tau_local[j] = mx;
                    atomicMin(reinterpret_cast<unsigned long long *>(a.tau_g + q0 + j),
                              (unsigned long long)mx);
                }
            }
            if (lane == 0) {
                uint64_t g = *reinterpret_cast<volatile uint64_t *>(a.tau_g + q0 + j);
                uint64_t t = S.tau_local[j];
                S.tau[j] = g < t ? g : t;
            }
        }
        __syncthreads();
    }

    // final cut to k', then append the survivors that beat the global bound
    for (int j = warp; j < QB && !a.keys_out; j += kWarps) {
        if (q0 + j >= a.B) continue;
        uint64_t *b = S.buf + (size_t)j * cap;
        int c = S.cnt[j];
        if (c > kp) {
            SelectResult sr = warp_select(b, c, kp, S.hist + warp * 256);
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
                uint64_t y = __shfl_xor_sync(0xffffffffu, mx, o);
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

// candidate buffer entries per query (none in dense-key mode)
inline int buffer_cap(const ScanArgs &a) { return a.keys_out ? 0 : a.kp + 2 * kRPI; }

template <int QB, bool BF>
cudaError_t launch_qb(const ScanArgs &a, int G, cudaStream_t s) {
    const int cap = buffer_cap(a);
    const size_t sm = smem_bytes(QB, a.ld, cap, BF);
    cudaError_t e = cudaFuncSetAttribute(scan_simt_kernel<QB, BF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((a.B + QB - 1) / QB, G);
    scan_simt_kernel<QB, BF><<<grid, kThreads, sm, s>>>(a, cap);
    return cudaGetLastError();
}

template <bool BF>
cudaError_t launch_bf(const ScanArgs &a, int QB, int G, cudaStream_t s) {
    switch (QB) {
        case 1: return launch_qb<1, BF>(a, G, s);
        case 2: return launch_qb<2, BF>(a, G, s);
        case 4: return launch_qb<4, BF>(a, G, s);
        case 8: return launch_qb<8, BF>(a, G, s);
        case 16: return launch_qb<16, BF>(a, G, s);
        default: return launch_qb<32, BF>(a, G, s);
    }
}


// ---------------------------------------------------------------------------
// Staged dense-key scan.  Same arithmetic and lane layout as the kernel
// above in dense-key mode, but the rows reach shared memory through bulk
// asynchronous copies (cp.async.bulk, one per row, completing on a stage
// mbarrier) issued by a producer warp, so the eight consumer warps never
// wait on global memory for row data and the copy engine keeps NS stages of
// 128 rows in flight.  Stage i holds chunk c0 + i (positions 128 c ..
// 128 c + 127 of the id list); row slots are padded by 64 bytes so that the
// consumers' 16-byte reads of eight rows are conflict-free.  Every wait is
// bounded (error word on timeout; the producer drains its copies before the
// CTA exits).
// ---------------------------------------------------------------------------
constexpr int kKCons = 256;                 // consumer threads
constexpr int kKThreads = kKCons + 32;      // + producer warp
constexpr int kKPad = 64;

struct KLayout {
    size_t q, qn, stage, ids, bar, total;
    int slot;
};

__host__ __device__ inline KLayout klayout(int QB, int ld, bool bf, int ns) {
    KLayout L;
    L.slot = ld * (bf ? 2 : 4) + kKPad;
    size_t o = 0;
    L.q = o;
    o += align16(qbytes(QB, ld, bf));
    L.qn = o;
    o += align16(QB * 4);
    o = (o + 127) & ~size_t(127);
    L.stage = o;
    o += (size_t)ns * kRPI * L.slot;
    L.ids = o;
    o += align16((size_t)ns * kRPI * 4);
    L.bar = o;
    o += align16((size_t)2 * ns * 8 + 8);
    L.total = o;
    return L;
}

__device__ __forceinline__ void bulk_row(uint32_t dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(umma::smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void cons_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kKCons) : "memory");
}
// Barrier over the consumer threads that also ORs a flag across them.
__device__ __forceinline__ bool cons_sync_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kKCons)
        : "memory");
    return r != 0;
}

template <int QB, bool BF>
__global__ void __launch_bounds__(kKThreads, 1)
scan_keys_staged_kernel(ScanArgs a, int ns) {
    constexpr int VEC = vec_of(BF);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ld = a.ld;
    const KLayout L = klayout(QB, ld, BF, ns);
    float *Qs = reinterpret_cast<float *>(smem_raw + L.q);
    float *qn = reinterpret_cast<float *>(smem_raw + L.qn);
    unsigned char *stages = smem_raw + L.stage;
    int32_t *sids = reinterpret_cast<int32_t *>(smem_raw + L.ids);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + L.bar), *empty = full + ns;
    __shared__ uint32_t cmin_s[2][QB];
    __shared__ int abort_s;
    volatile int *abort_flag = &abort_s;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q0 = blockIdx.x * QB;
    const int G = gridDim.y, g = blockIdx.y;
    const int64_t total = *a.count_dev;
    if (a.count_copy && blockIdx.x == 0 && threadIdx.x == 0) *a.count_copy = total;
    const int64_t nch = (total + kRPI - 1) / kRPI;
    const int64_t c0 = nch * g / G, c1 = nch * (g + 1) / G;
    const uint32_t row_bytes = (uint32_t)ld * (BF ? 2 : 4);

    if (tid == 0) {
        for (int i = 0; i < ns; ++i) {
            umma::mbar_init(&full[i], 1);
            umma::mbar_init(&empty[i], kKCons / 32);
        }
        abort_s = 0;
        umma::fence_mbar_init();
    }
    for (int j = tid; j < 2 * QB; j += kKThreads) cmin_s[j / QB][j % QB] = 0xffffffffu;
    __syncthreads();
    auto fail = [&]() {
        *abort_flag = 1;
        atomicExch(a.err, 1);
    };

    if (warp == kKCons / 32) {
        // ------------------------------------------------------------ producer
        int it = 0;
        bool ok = true;
        for (int64_t c = c0; c < c1; ++c, ++it) {
            const int st = it % ns;
            ok = __all_sync(0xffffffffu,
                            umma::mbar_wait(&empty[st], ((it / ns) & 1) ^ 1, abort_flag));
            if (!ok) break;
            const int64_t pos = c * kRPI + lane * 4;
            int32_t id[4];
            if (pos + 3 < total) {
                const int4 v = __ldg(reinterpret_cast<const int4 *>(a.ids + pos));
                id[0] = v.x;
                id[1] = v.y;
                id[2] = v.z;
                id[3] = v.w;
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r) id[r] = pos + r < total ? a.ids[pos + r] : -1;
            }
            *reinterpret_cast<int4 *>(sids + st * kRPI + lane * 4) = make_int4(id[0], id[1], id[2], id[3]);
            const int64_t left = total - c * kRPI;
            const uint32_t n_rows = (uint32_t)(left < kRPI ? left : kRPI);
            if (lane == 0) umma::mbar_expect_tx(&full[st], n_rows * row_bytes);
            __syncwarp();
            unsigned char *dst = stages + (size_t)st * kRPI * L.slot;
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (id[r] >= 0)
                    bulk_row(umma::smem_u32(dst + (size_t)(lane * 4 + r) * L.slot),
                             reinterpret_cast<const unsigned char *>(a.X) + (int64_t)id[r] * row_bytes,
                             row_bytes, &full[st]);
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&full[st]);
        }
        if (!ok) {
            if (lane == 0) {
                fail();
                // wait (bounded) for the copies of every stage still filling
                volatile int never = 0;
                for (int k = 1; k <= ns && it - k >= 0; ++k)
                    umma::mbar_wait(&full[(it - k) % ns], ((it - k) / ns) & 1, &never);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ consumers
        const int sub = lane & 3, slot = warp * 8 + (lane >> 2);
        const int steps = steps_of(ld, BF);
        const int span = steps * 4 * VEC;
        const int qreg = qregion(QB, ld, BF);
        for (int i = tid; i < QB * span; i += kKCons) {
            const int j = i / span, dd = i - j * span;
            const float v = (q0 + j < a.B && dd < ld) ? a.Q[(int64_t)(q0 + j) * ld + dd] : 0.0f;
            if constexpr (QB >= 2) {
                const int t = dd / (4 * VEC), s4 = (dd / VEC) & 3, ii = dd % VEC;
                Qs[s4 * qreg + (VEC * t + ii) * QB + j] = v;
            } else {
                Qs[dd] = v;
            }
        }
        for (int j = warp; j < QB; j += kKCons / 32) {
            float sq = 0.0f;
            if (q0 + j < a.B)
                for (int t = lane; t < ld; t += 32) {
                    const float v = a.Q[(int64_t)(q0 + j) * ld + t];
                    sq = fmaf(v, v, sq);
                }
            for (int o = 16; o; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
            if (lane == 0) qn[j] = sq;
        }
        cons_sync();
        constexpr int OWNK = QB >= 4 ? QB / 4 : QB;
        const int jb = QB >= 4 ? ((sub & 1) * 2 + (sub >> 1)) * (QB / 4) : 0;
        const float *Qr = Qs + sub * qreg;
        int it = 0;
        for (int64_t c = c0; c < c1; ++c, ++it) {
            const int st = it % ns;
            const bool okw = __all_sync(0xffffffffu, umma::mbar_wait(&full[st], (it / ns) & 1, abort_flag));
            // every consumer warp leaves together if any wait gave up
            if (cons_sync_or(!okw)) {
                if (!okw && lane == 0) fail();
                break;
            }
            int32_t row[kRPL];
            bool valid[kRPL];
            float xnr[kRPL];
#pragma unroll
            for (int r = 0; r < kRPL; ++r) {
                row[r] = sids[st * kRPI + slot + r * kSlots];
                valid[r] = row[r] >= 0;
                xnr[r] = (a.metric == 0 && valid[r]) ? __ldg(a.xnorm + row[r]) : 0.0f;
            }
            const unsigned char *xs = stages + (size_t)st * kRPI * L.slot;
            float acc[kRPL][QB];
            if constexpr (QB >= 2) {
                uint64_t acc2[kRPL][QB / 2];
#pragma unroll
                for (int r = 0; r < kRPL; ++r)
#pragma unroll
                    for (int j = 0; j < QB / 2; ++j) acc2[r][j] = 0ull;
                for (int t = 0; t < steps; ++t) {
                    // a step past the row (bf16 rows of an odd number of 16-element
                    // groups) reads zeros, not the slot padding
                    const bool in_row = t * 64 + sub * 16 < (int)row_bytes;
                    uint4 x[kRPL];
#pragma unroll
                    for (int r = 0; r < kRPL; ++r)
                        x[r] = in_row ? *reinterpret_cast<const uint4 *>(
                                            xs + (size_t)(slot + r * kSlots) * L.slot + t * 64 + sub * 16)
                                      : make_uint4(0, 0, 0, 0);
#pragma unroll
                    for (int i = 0; i < VEC; ++i) {
                        const uint64_t *qp = reinterpret_cast<const uint64_t *>(Qr + (VEC * t + i) * QB);
                        uint64_t qv[QB / 2];
#pragma unroll
                        for (int j = 0; j < QB / 2; ++j) qv[j] = qp[j];
#pragma unroll
                        for (int r = 0; r < kRPL; ++r) {
                            const uint64_t xx = pack2(elem<BF>(x[r], i));
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
                for (int t = 0; t < steps; ++t) {
                    const float *qd = Qs + t * 4 * VEC + sub * VEC;
                    const bool in_row = t * 64 + sub * 16 < (int)row_bytes;
#pragma unroll
                    for (int r = 0; r < kRPL; ++r) {
                        const uint4 x = in_row ? *reinterpret_cast<const uint4 *>(
                                                     xs + (size_t)(slot + r * kSlots) * L.slot + t * 64 + sub * 16)
                                               : make_uint4(0, 0, 0, 0);
#pragma unroll
                        for (int i = 0; i < VEC; ++i) acc[r][0] = fmaf(qd[i], elem<BF>(x, i), acc[r][0]);
                    }
                }
            }
            // the stage's rows are no longer needed
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&empty[st]);
            reduce4<QB>(acc, sub);

            uint32_t mn[OWNK];
#pragma unroll
            for (int jj = 0; jj < OWNK; ++jj) mn[jj] = 0xffffffffu;
            if (QB >= 4 || sub == 0) {
#pragma unroll
                for (int r = 0; r < kRPL; ++r) {
                    if (!valid[r]) continue;
                    const int64_t pos = c * kRPI + slot + r * kSlots;
#pragma unroll
                    for (int jj = 0; jj < OWNK; ++jj) {
                        const int j = jb + jj;
                        if (q0 + j >= a.B) continue;
                        const float dot = acc[r][jj];
                        const float key = a.metric == 0 ? fmaxf(qn[j] + xnr[r] - 2.0f * dot, 0.0f) : -dot;
                        a.keys_out[(int64_t)(q0 + j) * a.keys_ld + pos] = key;
                        mn[jj] = min(mn[jj], float_to_ordered(key));
                    }
                }
            }
            const int buf = it & 1;
#pragma unroll
            for (int jj = 0; jj < OWNK; ++jj) {
                mn[jj] = min(mn[jj], __shfl_xor_sync(0xffffffffu, mn[jj], 4));
                mn[jj] = min(mn[jj], __shfl_xor_sync(0xffffffffu, mn[jj], 8));
                mn[jj] = min(mn[jj], __shfl_xor_sync(0xffffffffu, mn[jj], 16));
                if (lane < 4 && (QB >= 4 || sub == 0) && q0 + jb + jj < a.B)
                    atomicMin(&cmin_s[buf][jb + jj], mn[jj]);
            }
            cons_sync();
            if (tid < QB) {
                if (q0 + tid < a.B) a.chunk_min[(int64_t)(q0 + tid) * a.cmin_ld + c] = cmin_s[buf][tid];
                cmin_s[buf][tid] = 0xffffffffu;   // reused two chunks later, after a barrier
            }
        }
    }
}

template <int QB, bool BF>
cudaError_t launch_staged_qb(const ScanArgs &a, int G, int ns, cudaStream_t s) {
    const size_t sm = klayout(QB, a.ld, BF, ns).total;
    cudaError_t e = cudaFuncSetAttribute(scan_keys_staged_kernel<QB, BF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((a.B + QB - 1) / QB, G);
    scan_keys_staged_kernel<QB, BF><<<grid, kKThreads, sm, s>>>(a, ns);
    return cudaGetLastError();
}

template <bool BF>
cudaError_t launch_staged_bf(const ScanArgs &a, int QB, int G, int ns, cudaStream_t s) {
    switch (QB) {
        case 1: return launch_staged_qb<1, BF>(a, G, ns, s);
        case 2: return launch_staged_qb<2, BF>(a, G, ns, s);
        case 4: return launch_staged_qb<4, BF>(a, G, ns, s);
        case 8: return launch_staged_qb<8, BF>(a, G, ns, s);
        case 16: return launch_staged_qb<16, BF>(a, G, ns, s);
        default: return launch_staged_qb<32, BF>(a, G, ns, s);
    }
}

// Stages that fit 200 KB of shared memory (0: the staged kernel does not fit).
int staged_stages(int QB, int ld, bool bf) {
    for (int ns = 4; ns >= 2; --ns)
        if (klayout(QB, ld, bf, ns).total <= (size_t)200 * 1024) return ns;
    return 0;
}

}  // namespace

// Queries per CTA for a batch of B (shared memory permitting; the launcher
// halves it until the kernel's shared memory fits).
int scan_simt_query_block(int B) {
    if (B <= 1) return 1;
    if (B <= 2) return 2;
    if (B <= 4) return 4;
    if (B <= 8) return 8;
    if (B <= 16) return 16;
    return 32;
}

size_t scan_simt_smem(int QB, int ld, int kp) { return smem_bytes(QB, ld, kp + 2 * kRPI, false); }

cudaError_t launch_scan_simt(const ScanArgs &a, int G, cudaStream_t s) {
    const bool bf = a.x_bf16 != 0;
    int QB = scan_simt_query_block(a.B);
    const int cap = buffer_cap(a);
    while (QB > 1 && smem_bytes(QB, a.ld, cap, bf) > 200 * 1024) QB >>= 1;
    if (smem_bytes(QB, a.ld, cap, bf) > 220 * 1024 || a.err == nullptr) return cudaErrorInvalidValue;
    return bf ? launch_bf<true>(a, QB, G, s) : launch_bf<false>(a, QB, G, s);
}

}  // namespace vrs

namespace vrs {

bool scan_keys_staged_fits(int B, int ld, int x_bf16) {
    return staged_stages(scan_simt_query_block(B), ld, x_bf16 != 0) > 0;
}

cudaError_t launch_scan_keys_staged(const ScanArgs &a, int G, cudaStream_t s) {
    const bool bf = a.x_bf16 != 0;
    const int QB = scan_simt_query_block(a.B);
    const int ns = staged_stages(QB, a.ld, bf);
    if (ns == 0 || a.keys_out == nullptr || a.ids == nullptr || a.count_dev == nullptr ||
        a.chunk_min == nullptr || a.err == nullptr)
        return cudaErrorInvalidValue;
    return bf ? launch_staged_bf<true>(a, QB, G, ns, s) : launch_staged_bf<false>(a, QB, G, ns, s);
}

}  // namespace vrs
