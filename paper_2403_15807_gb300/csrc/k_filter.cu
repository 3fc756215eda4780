// k_filter.cu -- relational predicate pushdown (Sec. 3.2).
//
// theta_R is a conjunction of half-open ranges on int32 attribute columns.
// Stage 1 (predicate): every row is tested once; each warp turns 128 rows
//   (one 16-byte load per lane per term) into four 32-bit bitmap words and
//   each 4096-row tile records how many rows it selected.
// Stage 2 (tile scan): exclusive prefix sum of the tile counts -> the output
//   offset of every tile, plus the total |sigma_theta(R)|.
// Stage 3 (compact): late materialisation of the selection as the ascending
//   list of qualifying row ids (Fig. 3, predicate-first strategy); each
//   thread owns one bitmap word, a block scan of word popcounts gives its
//   write position.
// Bit order: row i is bit (i % 32) of word (i / 32).
#include <algorithm>
#include <cstdint>

#include "vrs_internal.cuh"

namespace vrs {
namespace {

constexpr int kWordsPerTile = kTileRows / 32;   // 128
constexpr int kPredThreads = 256;               // 8 warps x 512 rows = 4096 rows

__device__ __forceinline__ bool in_range(int32_t a, int32_t lo, int32_t hi) {
    return lo <= a && a < hi;
}

// Grid: one block per 4096-row tile.
__global__ void __launch_bounds__(kPredThreads)
predicate_kernel(AttrArg attrs, int64_t n, PredArg p, uint32_t *__restrict__ bitmap,
                 int32_t *__restrict__ tile_counts) {
    __shared__ int32_t warp_cnt[kPredThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tile0 = (int64_t)blockIdx.x * kTileRows;
    int32_t cnt = 0;
    // each warp: 4 chunks of 128 rows; lane holds rows r0..r0+3
    for (int c = 0; c < 4; ++c) {
        const int64_t r0 = tile0 + (int64_t)warp * 512 + c * 128 + lane * 4;
        uint32_t nib = 0;
        if (r0 + 3 < n) {
            uint32_t m = 0xFu;
            for (int t = 0; t < p.n_terms; ++t) {
                int4 a = *reinterpret_cast<const int4 *>(attrs.col[p.col[t]] + r0);
                const int32_t lo = p.lo[t], hi = p.hi[t];
                m &= (uint32_t)in_range(a.x, lo, hi) | ((uint32_t)in_range(a.y, lo, hi) << 1) |
                     ((uint32_t)in_range(a.z, lo, hi) << 2) |
                     ((uint32_t)in_range(a.w, lo, hi) << 3);
            }
            nib = m;
        } else {
            for (int j = 0; j < 4; ++j) {
                const int64_t r = r0 + j;
                if (r >= n) break;
                bool ok = true;
                for (int t = 0; t < p.n_terms; ++t)
                    ok = ok && in_range(attrs.col[p.col[t]][r], p.lo[t], p.hi[t]);
                nib |= (uint32_t)ok << j;
            }
        }
        // gather 8 nibbles (lanes 8w..8w+7) into word w of this 128-row chunk
        uint32_t word = nib << (4 * (lane & 7));
        word |= __shfl_xor_sync(0xffffffffu, word, 1);
        word |= __shfl_xor_sync(0xffffffffu, word, 2);
        word |= __shfl_xor_sync(0xffffffffu, word, 4);
        if ((lane & 7) == 0) {
            const int64_t w = (r0 >> 5);
            if (w * 32 < n) bitmap[w] = word;
            cnt += __popc(word);
        }
    }
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) warp_cnt[warp] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t s = 0;
        for (int w = 0; w < kPredThreads / 32; ++w) s += warp_cnt[w];
        tile_counts[blockIdx.x] = s;
    }
}

// One block; exclusive scan of n_tiles int32 counts into int64 offsets.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads)
tile_scan_kernel(const int32_t *__restrict__ counts, int64_t n_tiles,
                 int64_t *__restrict__ offsets, int64_t *__restrict__ total) {
    __shared__ int64_t warp_sum[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t per = (n_tiles + kScanThreads - 1) / kScanThreads;
    const int64_t b = tid * per, e = min(n_tiles, b + per);
    int64_t local = 0;
    for (int64_t i = b; i < e; ++i) local += counts[i];
    int64_t incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t v = warp_sum[lane], x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        warp_sum[lane] = x - v;   // exclusive
        if (lane == 31) *total = x;
    }
    __syncthreads();
    int64_t run = warp_sum[warp] + incl - local;
    for (int64_t i = b; i < e; ++i) {
        offsets[i] = run;
        run += counts[i];
    }
}

// Grid: one block per tile, one thread per bitmap word.
__global__ void __launch_bounds__(kWordsPerTile)
compact_kernel(const uint32_t *__restrict__ bitmap, int64_t n,
               const int64_t *__restrict__ tile_offsets, int32_t *__restrict__ ids) {
    __shared__ int32_t warp_sum[kWordsPerTile / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t w = (int64_t)blockIdx.x * kWordsPerTile + tid;
    const int64_t n_words = (n + 31) / 32;
    uint32_t word = w < n_words ? bitmap[w] : 0u;
    int32_t c = __popc(word), incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    int32_t before = 0;
    for (int i = 0; i < warp; ++i) before += warp_sum[i];
    int64_t pos = tile_offsets[blockIdx.x] + before + incl - c;
    while (word) {
        int b = __ffs(word) - 1;
        word &= word - 1;
        ids[pos++] = (int32_t)(w * 32 + b);
    }
}

// Predicate straight to an (unordered) id list.  Each block takes
// kIdChunks consecutive 128-row chunks per warp; a warp tests 128 rows per
// chunk from 16-byte attribute loads (all chunks' loads issued up front),
// the block sums its warps' counts and reserves its output range with one
// atomic, and each warp writes its rows there.  Rows of one block stay
// ascending; blocks land in atomic order.  *count must be zero on entry.
constexpr int kIdChunks = 4;
__global__ void __launch_bounds__(256)
predicate_ids_kernel(AttrArg attrs, int64_t n, PredArg pv, const PredArg *__restrict__ pdev,
                     int32_t *__restrict__ ids, int64_t *__restrict__ count) {
    // a programmatically dependent distance pass may start its set-up now
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const PredArg p = pdev ? *pdev : pv;   // device copy when given (graph replays)
    __shared__ int warp_tot[8];
    __shared__ unsigned long long block_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t blk0 = (int64_t)blockIdx.x * 8 * kIdChunks * 128;
    // per term, the 16-byte loads of all chunks are issued together; a chunk
    // that runs past n (only in the last block) is tested row by row
    uint32_t nib[kIdChunks];
#pragma unroll
    for (int c = 0; c < kIdChunks; ++c) nib[c] = 0xFu;
    for (int t = 0; t < p.n_terms; ++t) {
        const int32_t *col = attrs.col[p.col[t]];
        const int32_t lo = p.lo[t], hi = p.hi[t];
        int4 v[kIdChunks];
#pragma unroll
        for (int c = 0; c < kIdChunks; ++c) {
            const int64_t r0 = blk0 + ((int64_t)warp * kIdChunks + c) * 128 + lane * 4;
            v[c] = r0 + 3 < n ? __ldg(reinterpret_cast<const int4 *>(col + r0)) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int c = 0; c < kIdChunks; ++c)
            nib[c] &= (uint32_t)in_range(v[c].x, lo, hi) | ((uint32_t)in_range(v[c].y, lo, hi) << 1) |
                      ((uint32_t)in_range(v[c].z, lo, hi) << 2) |
                      ((uint32_t)in_range(v[c].w, lo, hi) << 3);
    }
#pragma unroll
    for (int c = 0; c < kIdChunks; ++c) {
        const int64_t r0 = blk0 + ((int64_t)warp * kIdChunks + c) * 128 + lane * 4;
        if (r0 + 3 < n) continue;
        uint32_t m = 0;
        for (int j = 0; j < 4; ++j) {
            const int64_t r = r0 + j;
            if (r >= n) break;
            bool ok = true;
            for (int t = 0; t < p.n_terms; ++t)
                ok = ok && in_range(attrs.col[p.col[t]][r], p.lo[t], p.hi[t]);
            m |= (uint32_t)ok << j;
        }
        nib[c] = m;
    }
    // lane-major order inside the warp: chunk c, then lane
    int cl = 0;
#pragma unroll
    for (int c = 0; c < kIdChunks; ++c) cl += __popc(nib[c]);
    int incl = cl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < 8; ++w) tot += warp_tot[w];
        block_base = tot ? atomicAdd(reinterpret_cast<unsigned long long *>(count),
                                     (unsigned long long)tot)
                         : 0ull;
    }
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += warp_tot[w];
    int64_t o = (int64_t)block_base + before + incl - cl;
#pragma unroll
    for (int c = 0; c < kIdChunks; ++c) {
        const int64_t r0 = blk0 + ((int64_t)warp * kIdChunks + c) * 128 + lane * 4;
        for (int j = 0; j < 4; ++j)
            if ((nib[c] >> j) & 1u) ids[o++] = (int32_t)(r0 + j);
    }
}

// Rows r_i = floor(i n / M), i < M, that satisfy the predicate, appended in
// any order to ids (one atomic per warp).  *count must be zero on entry and
// ends at most M.
__global__ void __launch_bounds__(256)
sample_ids_kernel(AttrArg attrs, int64_t n, PredArg p, int64_t M, int32_t *__restrict__ ids,
                  int64_t *__restrict__ count) {
    const int lane = threadIdx.x & 31;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < M; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        const int64_t r = i < M ? i * n / M : 0;
        bool ok = i < M;
        for (int t = 0; t < p.n_terms && ok; ++t)
            ok = in_range(__ldg(attrs.col[p.col[t]] + r), p.lo[t], p.hi[t]);
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        unsigned long long base = 0;
        if (lane == 0 && bal)
            base = atomicAdd(reinterpret_cast<unsigned long long *>(count),
                             (unsigned long long)__popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (ok) ids[base + __popc(bal & ((1u << lane) - 1u))] = (int32_t)r;
    }
}

}  // namespace

cudaError_t launch_sample_ids(const AttrArg &attrs, int64_t n, const PredArg &p, int64_t M,
                              int32_t *ids, int64_t *count, cudaStream_t s) {
    if (M < 1 || M > n || n > INT32_MAX) return cudaErrorInvalidValue;
    const int64_t blocks = std::min<int64_t>(1024, (M + 255) / 256);
    sample_ids_kernel<<<(unsigned)blocks, 256, 0, s>>>(attrs, n, p, M, ids, count);
    return cudaGetLastError();
}

cudaError_t launch_predicate_ids(const AttrArg &attrs, int64_t n, const PredArg &p,
                                 const PredArg *pdev, int32_t *ids, int64_t *count, int n_sm,
                                 cudaStream_t s) {
    (void)n_sm;
    const int64_t rows_per_block = 8 * kIdChunks * 128;
    const int64_t blocks = (n + rows_per_block - 1) / rows_per_block;
    predicate_ids_kernel<<<(unsigned)std::max<int64_t>(1, blocks), 256, 0, s>>>(attrs, n, p, pdev,
                                                                                 ids, count);
    return cudaGetLastError();
}

cudaError_t launch_predicate(const AttrArg &attrs, int64_t n, const PredArg &p,
                             uint32_t *bitmap, int32_t *tile_counts, cudaStream_t s) {
    int64_t tiles = (n + kTileRows - 1) / kTileRows;
    predicate_kernel<<<(unsigned)tiles, kPredThreads, 0, s>>>(attrs, n, p, bitmap, tile_counts);
    return cudaGetLastError();
}

cudaError_t launch_tile_scan(const int32_t *tile_counts, int64_t n_tiles, int64_t *tile_offsets,
                             int64_t *total, cudaStream_t s) {
    tile_scan_kernel<<<1, kScanThreads, 0, s>>>(tile_counts, n_tiles, tile_offsets, total);
    return cudaGetLastError();
}

cudaError_t launch_compact(const uint32_t *bitmap, int64_t n, const int64_t *tile_offsets,
                           int32_t *ids, cudaStream_t s) {
    int64_t tiles = (n + kTileRows - 1) / kTileRows;
    compact_kernel<<<(unsigned)tiles, kWordsPerTile, 0, s>>>(bitmap, n, tile_offsets, ids);
    return cudaGetLastError();
}

}  // namespace vrs
