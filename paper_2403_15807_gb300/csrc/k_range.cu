// k_range.cu -- filtered range search: the selection sigma_eps of Sec. 3
// (eq. "Brute force similarity search with relational predicate theta") with
// eps a bound on the score.  Query b keeps every selected row whose squared
// L2 distance is <= eps (IP: q.x >= eps).
//
// It runs on the dense-key form of the GEMV plan: the distance pass has
// written every first-pass key of the query batch into a [B x rows] key
// matrix, with each query's minimum over every 128 positions.  Then:
//   mark  -- one CTA per query.  A chunk whose minimum exceeds the bound plus
//            a margin holds no result.  In the other chunks every position
//            whose first-pass key is within the margin of the bound gets its
//            exact FP32 score (direct form, as the re-rank computes it); the
//            key matrix keeps the exact score of each result and +inf
//            elsewhere, the chunk minimum becomes 0 (results) or ~0 (none),
//            and the query's result count is written.
//   write -- after the host has turned the counts into offsets: each result
//            is written at its query's offset (in no particular order).
// The margin bounds the difference between the first-pass key and the exact
// FP32 score, so every row whose exact score passes is examined.
#include "vrs_internal.cuh"

namespace vrs {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kChunk = 128;

__device__ __forceinline__ float finf() { return __int_as_float(0x7f800000); }

// Key-space bound: L2 keys are distances, IP keys are -q.x.
__device__ __forceinline__ float key_bound(int metric, float eps) {
    return metric == 0 ? eps : -eps;
}

__global__ void __launch_bounds__(1024) max_f32_kernel(const float *__restrict__ v, int64_t n,
                                                       float *__restrict__ out) {
    __shared__ float red[32];
    float m = 0.0f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, v[i]);
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) out[0] = m;
    }
}

__global__ void __launch_bounds__(kThreads) range_mark_kernel(RangeArgs a) {
    extern __shared__ float qs[];   // [ld] this query
    __shared__ float red[kWarps];
    __shared__ int64_t found_w[kWarps];
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < a.ld; i += kThreads) qs[i] = a.Q[(int64_t)b * a.ld + i];
    __syncthreads();
    float s2 = 0.0f;
    for (int i = tid; i < a.d; i += kThreads) s2 = fmaf(qs[i], qs[i], s2);
    for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (lane == 0) red[warp] = s2;
    __syncthreads();
    float qn = 0.0f;
    for (int w = 0; w < kWarps; ++w) qn += red[w];

    const int64_t count = *a.count_dev;
    const int64_t nch = (count + kChunk - 1) / kChunk;
    const float ekey = key_bound(a.metric, a.eps);
    // |first-pass key - exact FP32 score| stays below (8 d + 64) 2^-24 of
    // ||q||^2 + max ||x||^2: both sums of d terms carry at most ~d units of
    // rounding of that magnitude (the first pass's TF32 split adds less)
    const float margin = (8.0f * (float)a.d + 64.0f) * 5.9604645e-8f * (qn + *a.xn_max);
    const float T = ekey + margin;
    float *kb = a.keys + (int64_t)b * a.keys_ld;
    uint32_t *cm = a.chunk_min + (int64_t)b * a.cmin_ld;
    int64_t mine = 0;
    for (int64_t c = warp; c < nch; c += kWarps) {
        const uint32_t m = cm[c];
        if (m == 0xffffffffu || !(ordered_to_float(m) <= T)) {
            if (lane == 0) cm[c] = 0xffffffffu;
            continue;
        }
        int found = 0;
#pragma unroll 1
        for (int e = 0; e < kChunk / 32; ++e) {
            const int64_t p = c * kChunk + e * 32 + lane;
            const bool in = p < count;
            const float key = in ? kb[p] : finf();
            const bool cand = in && key <= T;
            float exact = finf();
            unsigned bal = __ballot_sync(0xffffffffu, cand);
            while (bal) {
                // the warp computes one candidate's exact score
                const int l = __ffs(bal) - 1;
                bal &= bal - 1;
                const int32_t id = a.ids[c * kChunk + e * 32 + l];
                const float *xr = a.X + (int64_t)id * a.ld;
                float acc = 0.0f;
                if (a.metric == 0) {
                    for (int t = lane; t < a.d; t += 32) {
                        const float df = qs[t] - xr[t];
                        acc = fmaf(df, df, acc);
                    }
                } else {
                    for (int t = lane; t < a.d; t += 32) acc = fmaf(qs[t], xr[t], acc);
                }
                for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == l) exact = a.metric == 0 ? acc : -acc;
            }
            if (in) {
                const bool pass = cand && exact <= ekey;
                kb[p] = pass ? exact : finf();
                found += pass;
            }
        }
        found = __reduce_add_sync(0xffffffffu, found);
        if (lane == 0) {
            cm[c] = found ? 0u : 0xffffffffu;
            mine += found;
        }
    }
    if (lane == 0) found_w[warp] = mine;
    __syncthreads();
    if (tid == 0) {
        int64_t total = 0;
        for (int w = 0; w < kWarps; ++w) total += found_w[w];
        a.counts[b] = total;
    }
}

__global__ void __launch_bounds__(kThreads) range_write_kernel(RangeArgs a) {
    __shared__ int slot;
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) slot = 0;
    __syncthreads();
    const int64_t count = *a.count_dev;
    const int64_t nch = (count + kChunk - 1) / kChunk;
    const float ekey = key_bound(a.metric, a.eps);
    const int64_t base = a.offsets[b], limit = a.offsets[b + 1] - base;
    const float *kb = a.keys + (int64_t)b * a.keys_ld;
    const uint32_t *cm = a.chunk_min + (int64_t)b * a.cmin_ld;
    for (int64_t c = warp; c < nch; c += kWarps) {
        if (cm[c] != 0u) continue;
        for (int e = 0; e < kChunk / 32; ++e) {
            const int64_t p = c * kChunk + e * 32 + lane;
            const bool in = p < count;
            const float key = in ? kb[p] : finf();
            const bool pass = in && key <= ekey;
            const unsigned bal = __ballot_sync(0xffffffffu, pass);
            if (!bal) continue;
            int w = 0;
            if (lane == 0) w = atomicAdd(&slot, __popc(bal));
            w = __shfl_sync(0xffffffffu, w, 0);
            if (pass) {
                const int64_t o = w + __popc(bal & ((1u << lane) - 1u));
                if (o < limit) {
                    a.out_ids[base + o] = a.ids[p];
                    a.out_dist[base + o] = a.metric == 0 ? key : -key;
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_max_f32(const float *v, int64_t n, float *out, cudaStream_t s) {
    if (!v || !out || n < 1) return cudaErrorInvalidValue;
    max_f32_kernel<<<1, 1024, 0, s>>>(v, n, out);
    return cudaGetLastError();
}

cudaError_t launch_range_mark(const RangeArgs &a, cudaStream_t s) {
    if (a.B < 1 || !a.keys || !a.chunk_min || !a.ids || !a.count_dev || !a.X || !a.Q ||
        !a.xn_max || !a.counts || a.ld < a.d || a.ld > 12 * 1024)
        return cudaErrorInvalidValue;
    range_mark_kernel<<<a.B, kThreads, (size_t)a.ld * 4, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_range_write(const RangeArgs &a, cudaStream_t s) {
    if (a.B < 1 || !a.keys || !a.chunk_min || !a.ids || !a.count_dev || !a.offsets ||
        !a.out_ids || !a.out_dist)
        return cudaErrorInvalidValue;
    range_write_kernel<<<a.B, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace vrs
