// k_load.cu -- load-time work on the vector column (off the query path).
//
// The paper normalises and (re)materialises per query inside the Tensor
// pipeline (Sec. 5.2: filter -> materialise -> normalise -> dot product);
// here the per-row quantities are computed once when the column is loaded:
//   * a row-padded float32 or bf16 copy (row stride a multiple of 16
//     elements so every row starts 64-byte aligned for vector loads / TMA);
//   * ||x_i||^2 in float32 with compensated (Neumaier) summation of exactly
//     split squares, for the L2 expansion ||q||^2 - 2 q.x + ||x||^2;
//   * reduced-precision copies: bf16 (round to nearest even) and FP8 E4M3
//     with one float32 scale per row (scale = max|x| / 448).
// One warp per row, rows in a grid-stride loop.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "vrs_internal.cuh"

namespace vrs {
namespace {

constexpr int kWarps = 8;

__device__ __forceinline__ int64_t warp_row0() {
    return (int64_t)blockIdx.x * kWarps + threadIdx.x / 32;
}
__device__ __forceinline__ int64_t warp_rows_step() { return (int64_t)gridDim.x * kWarps; }

__global__ void copy_f32_kernel(const float *__restrict__ src, int64_t n, int32_t d,
                                float *__restrict__ dst, int32_t ld) {
    int lane = threadIdx.x & 31;
    for (int64_t r = warp_row0(); r < n; r += warp_rows_step())
        for (int t = lane; t < ld; t += 32) dst[r * ld + t] = t < d ? src[r * d + t] : 0.0f;
}

// dst row i = src row ids[i] (float32, d values per row)
__global__ void gather_rows_f32_kernel(const float *__restrict__ src, int32_t d,
                                       const int32_t *__restrict__ ids, int64_t m,
                                       float *__restrict__ dst) {
    int lane = threadIdx.x & 31;
    for (int64_t r = warp_row0(); r < m; r += warp_rows_step()) {
        const float *s = src + (int64_t)ids[r] * d;
        for (int t = lane; t < d; t += 32) dst[r * d + t] = s[t];
    }
}

__global__ void bf16_to_f32_kernel(const uint16_t *__restrict__ src, int64_t n, int32_t d,
                                   float *__restrict__ dst, int32_t ld) {
    int lane = threadIdx.x & 31;
    for (int64_t r = warp_row0(); r < n; r += warp_rows_step())
        for (int t = lane; t < ld; t += 32) {
            float v = 0.0f;
            if (t < d) v = __uint_as_float((uint32_t)src[r * d + t] << 16);
            dst[r * ld + t] = v;
        }
}

__global__ void copy_bf16_kernel(const uint16_t *__restrict__ src, int64_t n, int32_t d,
                                 uint16_t *__restrict__ dst, int32_t ld) {
    int lane = threadIdx.x & 31;
    for (int64_t r = warp_row0(); r < n; r += warp_rows_step())
        for (int t = lane; t < ld; t += 32) dst[r * ld + t] = t < d ? src[r * d + t] : 0;
}

__global__ void f32_to_bf16_kernel(const float *__restrict__ src, int64_t n, int32_t d,
                                   int32_t lds, uint16_t *__restrict__ dst, int32_t ld) {
    int lane = threadIdx.x & 31;
    for (int64_t r = warp_row0(); r < n; r += warp_rows_step())
        for (int t = lane; t < ld; t += 32) {
            __nv_bfloat16 h = __float2bfloat16_rn(t < d ? src[r * lds + t] : 0.0f);
            dst[r * ld + t] = __bfloat16_as_ushort(h);
        }
}

// Pair copy of float32 rows: dst row r = [x1 (ldp values) | x2 (ldp values)]
// with x1 = bf16(x), x2 = bf16(x - x1) (round to nearest even), zero past d.
__global__ void f32_to_pair_kernel(const float *__restrict__ src, int64_t n, int32_t d,
                                   int32_t lds, uint16_t *__restrict__ dst, int32_t ldp) {
    int lane = threadIdx.x & 31;
    for (int64_t r = warp_row0(); r < n; r += warp_rows_step())
        for (int t = lane; t < ldp; t += 32) {
            const float v = t < d ? src[r * lds + t] : 0.0f;
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
            dst[r * 2 * ldp + t] = __bfloat16_as_ushort(h);
            dst[r * 2 * ldp + ldp + t] = __bfloat16_as_ushort(l);
        }
}

__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__global__ void f32_to_e4m3_kernel(const float *__restrict__ src, int64_t n, int32_t d,
                                   int32_t lds, uint8_t *__restrict__ dst, int32_t ld,
                                   float *__restrict__ scale) {
    int lane = threadIdx.x & 31;
    for (int64_t r = warp_row0(); r < n; r += warp_rows_step()) {
        float amax = 0.0f;
        for (int t = lane; t < d; t += 32) amax = fmaxf(amax, fabsf(src[r * lds + t]));
        amax = warp_max(amax);
        float s = amax > 0.0f ? __fdiv_rn(amax, 448.0f) : 1.0f;
        if (lane == 0) scale[r] = s;
        for (int t = lane; t < ld; t += 32) {
            uint8_t c = 0;
            if (t < d) {
                float v = __fdiv_rn(src[r * lds + t], s);
                c = (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
            }
            dst[r * ld + t] = c;
        }
    }
}

// Neumaier accumulation of a sum of squares.  Each square is split exactly
// into p + e (p = fl(v*v), e = fma(v, v, -p)); p goes through the
// compensated sum, e into the compensation term.
struct Comp {
    float s, c;
};
__device__ __forceinline__ void comp_add(Comp &a, float v) {
    float t = a.s + v;
    if (fabsf(a.s) >= fabsf(v)) a.c += (a.s - t) + v;
    else a.c += (v - t) + a.s;
    a.s = t;
}
__device__ __forceinline__ void comp_add_sq(Comp &a, float x) {
    float p = x * x;
    float e = fmaf(x, x, -p);
    comp_add(a, p);
    a.c += e;
}
__device__ __forceinline__ float comp_warp_total(Comp a) {
    for (int o = 16; o; o >>= 1) {
        float s2 = __shfl_xor_sync(0xffffffffu, a.s, o);
        float c2 = __shfl_xor_sync(0xffffffffu, a.c, o);
        a.c += c2;
        comp_add(a, s2);
    }
    return a.s + a.c;
}

__global__ void norms_f32_kernel(const float *__restrict__ x, int64_t n, int32_t d, int32_t ld,
                                 float *__restrict__ out) {
    int lane = threadIdx.x & 31;
    for (int64_t r = warp_row0(); r < n; r += warp_rows_step()) {
        Comp a{0.0f, 0.0f};
        for (int t = lane; t < d; t += 32) comp_add_sq(a, x[r * ld + t]);
        float v = comp_warp_total(a);
        if (lane == 0) out[r] = v;
    }
}

__global__ void norms_bf16_kernel(const uint16_t *__restrict__ x, int64_t n, int32_t d,
                                  int32_t ld, float *__restrict__ out) {
    int lane = threadIdx.x & 31;
    for (int64_t r = warp_row0(); r < n; r += warp_rows_step()) {
        Comp a{0.0f, 0.0f};
        for (int t = lane; t < d; t += 32) comp_add_sq(a, __uint_as_float((uint32_t)x[r * ld + t] << 16));
        float v = comp_warp_total(a);
        if (lane == 0) out[r] = v;
    }
}

__global__ void prep_queries_kernel(const float *__restrict__ q, int32_t B, int32_t d,
                                    float *__restrict__ qpad, int32_t ld,
                                    uint64_t *__restrict__ tau_g, int32_t *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = warp_row0(); r < B; r += warp_rows_step()) {
        for (int t = lane; t < ld; t += 32) qpad[r * ld + t] = t < d ? q[r * d + t] : 0.0f;
        if (lane == 0) {
            if (tau_g) tau_g[r] = kEmpty;
            if (cnt) cnt[r] = 0;
        }
    }
}

// Decoded value of an E4M3 code (the library's conversion intrinsic).
__device__ __forceinline__ float e4m3_value(uint8_t c) {
    const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)c, __NV_E4M3);
    return __half2float(__half(h));
}

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One warp per query row: encode to the tensor operand type; qres[r] (if
// set) = ||q - decoded encoding|| in float64, rounded up to float.
__global__ void prep_tensor_queries_kernel(const float *__restrict__ qpad, int32_t B,
                                           int32_t Bpad, int32_t d, int32_t ld, int dtype,
                                           unsigned char *__restrict__ Qenc, int32_t row_bytes,
                                           float *__restrict__ qnorm, float *__restrict__ qscale,
                                           float *__restrict__ qres) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = warp_row0(); r < Bpad; r += warp_rows_step()) {
        unsigned char *dst = Qenc + r * row_bytes;
        if (r >= B) {
            for (int i = lane; i < row_bytes; i += 32) dst[i] = 0;
            continue;
        }
        const float *src = qpad + r * ld;
        float ss = 0.0f;
        for (int t = lane; t < d; t += 32) ss = fmaf(src[t], src[t], ss);
        for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) qnorm[r] = ss;
        double res = 0.0;
        if (dtype == 1) {
            uint16_t *h = reinterpret_cast<uint16_t *>(dst);
            for (int t = lane; t < row_bytes / 2; t += 32) {
                const __nv_bfloat16 b = __float2bfloat16_rn(t < d ? src[t] : 0.0f);
                h[t] = t < d ? __bfloat16_as_ushort(b) : 0;
                if (t < d) {
                    const double e = (double)src[t] - (double)__bfloat162float(b);
                    res += e * e;
                }
            }
        } else {
            float amax = 0.0f;
            for (int t = lane; t < d; t += 32) amax = fmaxf(amax, fabsf(src[t]));
            amax = warp_max(amax);
            const float sc = amax > 0.0f ? __fdiv_rn(amax, 448.0f) : 1.0f;
            if (lane == 0) qscale[r] = sc;
            for (int t = lane; t < row_bytes; t += 32) {
                unsigned char c = 0;
                if (t < d) {
                    c = (unsigned char)__nv_cvt_float_to_fp8(__fdiv_rn(src[t], sc), __NV_SATFINITE,
                                                             __NV_E4M3);
                    const double e = (double)src[t] - (double)sc * (double)e4m3_value(c);
                    res += e * e;
                }
                dst[t] = c;
            }
        }
        res = warp_sum_d(res);
        if (qres && lane == 0) qres[r] = __double2float_ru(sqrt(res) * (1.0 + 1e-12));
    }
}

// Per-row norm and encoding residual, max over the rows (float bits of
// non-negative floats order like unsigned integers).
__global__ void encoding_stats_kernel(const float *__restrict__ x, int64_t n, int32_t d,
                                      int32_t ld, int dtype, const uint16_t *__restrict__ xb,
                                      const uint8_t *__restrict__ x8,
                                      const float *__restrict__ s8, float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    float mx_norm = 0.0f, mx_res = 0.0f;
    for (int64_t r = warp_row0(); r < n; r += warp_rows_step()) {
        double nn = 0.0, rr = 0.0;
        const double sc = (dtype == 2 && s8) ? (double)s8[r] : 1.0;
        for (int t = lane; t < d; t += 32) {
            const double v = (double)x[r * ld + t];
            nn += v * v;
            double dec = v;
            if (dtype == 1 && xb) dec = (double)__uint_as_float((uint32_t)xb[r * ld + t] << 16);
            else if (dtype == 2 && x8) dec = sc * (double)e4m3_value(x8[r * ld + t]);
            const double e = v - dec;
            rr += e * e;
        }
        nn = warp_sum_d(nn);
        rr = warp_sum_d(rr);
        mx_norm = fmaxf(mx_norm, __double2float_ru(sqrt(nn) * (1.0 + 1e-12)));
        mx_res = fmaxf(mx_res, __double2float_ru(sqrt(rr) * (1.0 + 1e-12)));
    }
    if (lane == 0) {
        atomicMax(reinterpret_cast<unsigned int *>(out), __float_as_uint(mx_norm));
        atomicMax(reinterpret_cast<unsigned int *>(out + 1), __float_as_uint(mx_res));
    }
}

__global__ void cert_seed_kernel(const float *__restrict__ dup, const float *__restrict__ qnorm,
                                 CertArgs c, int metric, int32_t B, uint64_t *__restrict__ tau_g,
                                 int32_t *__restrict__ cnt) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    // |q| from the pass's own float32 sum of squares, rounded up past its
    // accumulation error
    const float qn = sqrtf(fmaxf(qnorm[b], 0.0f) * (1.0f + (float)(c.d + 4) * 5.9604645e-08f)) *
                     1.0000002f;
    const float rq = c.rq ? c.rq[b] : 0.0f;
    const float T = dup[b] + cert_bound(qn, rq, c, metric);
    tau_g[b] = ((uint64_t)float_to_ordered(T) << 32) | 0xffffffffull;
    cnt[b] = 0;
}

int rows_grid(int64_t n) {
    int64_t g = (n + kWarps - 1) / kWarps;
    if (g > 152 * 64) g = 152 * 64;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_copy_f32(const float *src, int64_t n, int32_t d, float *dst, int32_t ld,
                            cudaStream_t s) {
    copy_f32_kernel<<<rows_grid(n), kWarps * 32, 0, s>>>(src, n, d, dst, ld);
    return cudaGetLastError();
}
cudaError_t launch_bf16_to_f32(const uint16_t *src, int64_t n, int32_t d, float *dst,
                               int32_t ld, cudaStream_t s) {
    bf16_to_f32_kernel<<<rows_grid(n), kWarps * 32, 0, s>>>(src, n, d, dst, ld);
    return cudaGetLastError();
}
cudaError_t launch_copy_bf16(const uint16_t *src, int64_t n, int32_t d, uint16_t *dst,
                             int32_t ld, cudaStream_t s) {
    copy_bf16_kernel<<<rows_grid(n), kWarps * 32, 0, s>>>(src, n, d, dst, ld);
    return cudaGetLastError();
}
cudaError_t launch_f32_to_bf16(const float *src, int64_t n, int32_t d, int32_t lds,
                               uint16_t *dst, int32_t ld, cudaStream_t s) {
    f32_to_bf16_kernel<<<rows_grid(n), kWarps * 32, 0, s>>>(src, n, d, lds, dst, ld);
    return cudaGetLastError();
}
cudaError_t launch_f32_to_pair(const float *src, int64_t n, int32_t d, int32_t lds,
                               uint16_t *dst, int32_t ldp, cudaStream_t s) {
    if (!src || !dst || n < 1 || d < 1 || ldp < d || ldp % 64) return cudaErrorInvalidValue;
    f32_to_pair_kernel<<<rows_grid(n), kWarps * 32, 0, s>>>(src, n, d, lds, dst, ldp);
    return cudaGetLastError();
}
cudaError_t launch_f32_to_e4m3(const float *src, int64_t n, int32_t d, int32_t lds,
                               uint8_t *dst, int32_t ld, float *scale, cudaStream_t s) {
    f32_to_e4m3_kernel<<<rows_grid(n), kWarps * 32, 0, s>>>(src, n, d, lds, dst, ld, scale);
    return cudaGetLastError();
}
cudaError_t launch_gather_rows_f32(const float *src, int32_t d, const int32_t *ids, int64_t m,
                                   float *dst, cudaStream_t s) {
    if (!src || !ids || !dst || m < 1 || d < 1) return cudaErrorInvalidValue;
    gather_rows_f32_kernel<<<rows_grid(m), kWarps * 32, 0, s>>>(src, d, ids, m, dst);
    return cudaGetLastError();
}
cudaError_t launch_prep_queries(const float *q, int32_t B, int32_t d, float *qpad, int32_t ld,
                                uint64_t *tau_g, int32_t *cand_cnt, cudaStream_t s) {
    prep_queries_kernel<<<rows_grid(B), kWarps * 32, 0, s>>>(q, B, d, qpad, ld, tau_g, cand_cnt);
    return cudaGetLastError();
}
cudaError_t launch_prep_tensor_queries(const float *qpad, int32_t B, int32_t Bpad, int32_t d,
                                       int32_t ld, int dtype, unsigned char *Qenc,
                                       int32_t row_bytes, float *qnorm, float *qscale,
                                       float *qres, cudaStream_t s) {
    prep_tensor_queries_kernel<<<rows_grid(Bpad), kWarps * 32, 0, s>>>(
        qpad, B, Bpad, d, ld, dtype, Qenc, row_bytes, qnorm, qscale, qres);
    return cudaGetLastError();
}
cudaError_t launch_encoding_stats(const float *x, int64_t n, int32_t d, int32_t ld, int dtype,
                                  const uint16_t *xb, const uint8_t *x8, const float *s8,
                                  float *out, cudaStream_t s) {
    if (!x || !out || n < 1 || d < 1 || ld < d || (dtype == 1 && !xb) ||
        (dtype == 2 && (!x8 || !s8)))
        return cudaErrorInvalidValue;
    encoding_stats_kernel<<<rows_grid(n), kWarps * 32, 0, s>>>(x, n, d, ld, dtype, xb, x8, s8, out);
    return cudaGetLastError();
}
cudaError_t launch_cert_seed(const float *dup, const float *qnorm, CertArgs c, int metric,
                             int32_t B, uint64_t *tau_g, int32_t *cnt, cudaStream_t s) {
    if (!dup || !qnorm || !tau_g || !cnt || B < 1) return cudaErrorInvalidValue;
    cert_seed_kernel<<<(B + 127) / 128, 128, 0, s>>>(dup, qnorm, c, metric, B, tau_g, cnt);
    return cudaGetLastError();
}
cudaError_t launch_norms_f32(const float *x, int64_t n, int32_t d, int32_t ld, float *out,
                             cudaStream_t s) {
    norms_f32_kernel<<<rows_grid(n), kWarps * 32, 0, s>>>(x, n, d, ld, out);
    return cudaGetLastError();
}
cudaError_t launch_norms_bf16(const uint16_t *x, int64_t n, int32_t d, int32_t ld, float *out,
                              cudaStream_t s) {
    norms_bf16_kernel<<<rows_grid(n), kWarps * 32, 0, s>>>(x, n, d, ld, out);
    return cudaGetLastError();
}

}  // namespace vrs
