// k_probe.cu -- a measurement kernel, not part of the query path: the rate at
// which this GPU reads whole rows at listed positions of a row-major table,
// the access pattern of the distance pass over a selection (every selected
// row read once, in full).  One warp instruction reads 512 contiguous bytes
// of a row (16 per lane).  Warp w of W takes list entries w, w + W, w + 2W,
// ..., eight at a time, so every warp has eight rows' loads in flight and a
// partial last pass over the list is spread over all warps; three 512-thread blocks per SM
// (~190 KB of row loads in flight per SM).
// The values read are summed (one atomic per block), so no load is dead.
#include <algorithm>

#include "vrs_internal.cuh"

namespace vrs {
namespace {

constexpr int kProbeThreads = 512;
constexpr int kProbeRows = 8;   // rows in flight per warp

__global__ void __launch_bounds__(kProbeThreads, 3)
gather_probe_kernel(const uint4 *__restrict__ X, int64_t n_rows, int64_t row_vec,
                    const int32_t *__restrict__ ids, int64_t m, float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * kProbeThreads + threadIdx.x) >> 5;
    const int64_t W = ((int64_t)gridDim.x * kProbeThreads) >> 5;
    float acc = 0.0f;
    for (int64_t r0 = w; r0 < m; r0 += W * kProbeRows) {
        int32_t id[kProbeRows];
#pragma unroll
        for (int u = 0; u < kProbeRows; ++u) {
            const int64_t r = r0 + (int64_t)u * W;
            const int32_t v = r < m ? __ldg(ids + r) : -1;
            id[u] = v < n_rows ? v : -1;   // ids outside the table are skipped
        }
        for (int64_t v0 = 0; v0 < row_vec; v0 += 32) {
            uint4 x[kProbeRows];
#pragma unroll
            for (int u = 0; u < kProbeRows; ++u)
                x[u] = (id[u] >= 0 && v0 + lane < row_vec) ? __ldg(X + (int64_t)id[u] * row_vec + v0 + lane)
                                                          : make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int u = 0; u < kProbeRows; ++u)
                acc += __uint_as_float(x[u].x) + __uint_as_float(x[u].y) + __uint_as_float(x[u].z) +
                       __uint_as_float(x[u].w);
        }
    }
    // one atomic per block (per-warp atomics on one word serialise at the end)
    __shared__ float ws[kProbeThreads / 32];
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < kProbeThreads / 32 ? ws[threadIdx.x] : 0.0f;
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) atomicAdd(out, acc);
    }
}

}  // namespace

cudaError_t launch_gather_probe(const void *rows, int64_t n_rows, int64_t row_bytes,
                                const int32_t *ids, int64_t m, float *out, int n_sm, cudaStream_t s) {
    if (!rows || !out || (m > 0 && !ids) || m < 0 || n_rows < 0 || row_bytes < 16 || row_bytes % 16 ||
        reinterpret_cast<uintptr_t>(rows) % 16)
        return cudaErrorInvalidValue;
    gather_probe_kernel<<<(unsigned)std::max(1, 3 * n_sm), kProbeThreads, 0, s>>>(
        static_cast<const uint4 *>(rows), n_rows, row_bytes / 16, ids, m, out);
    return cudaGetLastError();
}

}  // namespace vrs
