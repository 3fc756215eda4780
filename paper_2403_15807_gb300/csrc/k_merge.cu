// k_merge.cu -- cross-CTA merge of the per-CTA candidates, exact FP32
// re-rank, and the final per-query top-k (sorted by distance, ties by the
// smaller id; padded with id -1 / +inf).
//
// One CTA per query.  (1) A block radix select over the query's G*k'
// composites (read from L2) picks the k' best first-pass candidates.
// (2) Each warp recomputes the exact distance of one candidate at a time
// from the re-rank copy (float32 master, or the stored bf16 values):
// L2 in the direct form sum_t (q_t - x_t)^2, IP as q.x -- the form the
// definition uses (Sec. 3, eq. "Brute force similarity search with
// relational predicate"), which avoids the cancellation of the expanded
// ||q||^2 - 2 q.x + ||x||^2 used by the first pass.  (3) A bitonic sort of
// the k' exact composites in shared memory; the first k are written out.
#include <algorithm>

#include "topk_select.cuh"
#include "vrs_internal.cuh"

namespace vrs {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float load_master(const MergeArgs &a, int64_t off) {
    return a.Xf ? __ldg(a.Xf + off) : __uint_as_float((uint32_t)__ldg(a.Xb + off) << 16);
}

__global__ void __launch_bounds__(kThreads)
merge_rerank_kernel(MergeArgs a, int sort_n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sel = reinterpret_cast<uint64_t *>(smem_raw);              // [sort_n]
    uint64_t *stg = sel + sort_n;                                         // [stage_cap]
    float *qs = reinterpret_cast<float *>(stg + a.stage_cap);            // [ldq]
    __shared__ int hist[256];
    __shared__ int scratch[4];
    __shared__ int n_sel;

    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t mq = a.cand_cnt ? (int64_t)a.cand_cnt[b] : a.m;
    const uint64_t *cand = a.cand + (int64_t)b * a.m;
    // candidates that fit are staged in shared memory: the radix select then
    // makes its passes there instead of over L2
    if (mq <= a.stage_cap) {
        for (int64_t i = tid; i < mq; i += kThreads) stg[i] = cand[i];
        cand = stg;
        __syncthreads();
    }
    const int kq = a.k ? a.k[b] : a.k_shared;

    // number of non-empty candidates
    if (tid == 0) n_sel = 0;
    for (int i = tid; i < a.ldq; i += kThreads) qs[i] = a.Q[(int64_t)b * a.ldq + i];
    __syncthreads();
    int nv = 0;
    for (int64_t i = tid; i < mq; i += kThreads) nv += cand[i] != kEmpty;
    for (int o = 16; o; o >>= 1) nv += __shfl_xor_sync(0xffffffffu, nv, o);
    if (lane == 0) atomicAdd(&n_sel, nv);
    __syncthreads();
    const int n_valid = n_sel;
    const int want = min(a.kp, n_valid);
    __syncthreads();
    if (tid == 0) n_sel = 0;
    __syncthreads();

    // (1) the `want` best first-pass candidates
    SelectResult sr{~0ull, 0ull};   // keeps everything
    if (want < n_valid) sr = block_select(cand, mq, want, hist, scratch);
    for (int64_t i = tid; i < mq; i += kThreads) {
        uint64_t x = cand[i];
        if (x != kEmpty && sel_keep(x, sr)) {
            int p = atomicAdd(&n_sel, 1);
            sel[p] = x;
        }
    }
    __syncthreads();
    const int ns = n_sel;   // == want
    for (int i = ns + tid; i < sort_n; i += kThreads) sel[i] = kEmpty;
    __syncthreads();

    // (2) exact re-rank
    if (a.rerank) {
        for (int i = warp; i < ns; i += kThreads / 32) {
            const int32_t id = (int32_t)(sel[i] & 0xffffffffu);
            const int64_t off = (int64_t)id * a.ld;
            float acc = 0.0f;
            if (a.metric == 0) {
                for (int t = lane; t < a.d; t += 32) {
                    float df = qs[t] - load_master(a, off + t);
                    acc = fmaf(df, df, acc);
                }
            } else {
                for (int t = lane; t < a.d; t += 32) acc = fmaf(qs[t], load_master(a, off + t), acc);
            }
            for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) sel[i] = make_cand(a.metric == 0 ? acc : -acc, id);
        }
        __syncthreads();
    }

    // (3) bitonic sort of sel[0..sort_n)
    for (int size = 2; size <= sort_n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < sort_n / 2; i += kThreads) {
                int lo = 2 * i - (i & (stride - 1));
                int hi = lo + stride;
                bool up = (lo & size) == 0;
                uint64_t x = sel[lo], y = sel[hi];
                if ((x > y) == up) {
                    sel[lo] = y;
                    sel[hi] = x;
                }
            }
            __syncthreads();
        }
    }

    for (int i = tid; i < a.k_max; i += kThreads) {
        int64_t id = -1;
        float dist = __int_as_float(0x7f800000);
        if (i < kq && i < ns) {
            uint64_t c = sel[i];
            id = (int64_t)(c & 0xffffffffu);
            float key = ordered_to_float((uint32_t)(c >> 32));
            dist = a.metric == 0 ? key : -key;
        }
        a.out_ids[(int64_t)b * a.k_max + i] = id;
        a.out_dist[(int64_t)b * a.k_max + i] = dist;
    }
    // leave the per-query search state cleared for the next query
    if (a.reset_tau && tid == 0) {
        a.reset_tau[b] = kEmpty;
        if (a.cand_cnt) const_cast<int32_t *>(a.cand_cnt)[b] = 0;
    }
    if (a.reset_count && tid == 0 && b == 0) *a.reset_count = 0;
}

constexpr int kChunkKeys = 3072;   // keys per chunk
constexpr int kSample = 256;       // strided sample of a chunk for the pre-filter

// Block (p, b): the k' best of partition p of query b's keys, chunk by
// chunk.  Per chunk: (1) one warp takes the k'-th best of a strided sample of
// 256 keys plus the k' best so far -- an upper bound on the chunk's k'-th
// best; (2) every key at or below it is appended to a short list (few:
// about k' * chunk / sample); (3) one warp keeps the k' best of that list.
__global__ void __launch_bounds__(kThreads)
keys_topk_kernel(KeysTopkArgs a) {
    // k' best so far, then the chunk's survivors: at most k' + one chunk
    __shared__ uint64_t cand[kMaxKp + kChunkKeys];
    __shared__ uint64_t samp[kSample + kMaxKp];
    __shared__ int hist[256];
    __shared__ int n_cand, base;
    __shared__ uint64_t thr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b = blockIdx.y, P = gridDim.x, p = blockIdx.x;
    const int kp = a.kp;
    const int64_t count = a.count_dev ? *a.count_dev : a.n_pos;
    const int64_t beg = count * p / P, end = count * (p + 1) / P;
    const float *kb = a.keys + (int64_t)b * a.ld;
    auto comp = [&](int64_t pos) -> uint64_t {
        const float key = kb[pos];
        if (!(key < __int_as_float(0x7f800000))) return kEmpty;
        return make_cand(key, a.ids ? a.ids[pos] : (int32_t)pos);
    };
    int best = 0;
    for (int64_t c0 = beg; c0 < end; c0 += kChunkKeys) {
        const int m = (int)(end - c0 < kChunkKeys ? end - c0 : kChunkKeys);
        // (1) threshold from a strided sample plus the current best
        const int stride = m > kSample ? m / kSample : 1;
        const int ns = m > kSample ? kSample : m;
        for (int i = tid; i < ns; i += kThreads) samp[i] = comp(c0 + (int64_t)i * stride);
        for (int i = tid; i < best; i += kThreads) samp[ns + i] = cand[i];
        __syncthreads();
        if (warp == 0) {
            const int tot = ns + best;
            int nv = 0;
            for (int i = lane; i < tot; i += 32) nv += samp[i] != kEmpty;
#pragma unroll
            for (int o = 16; o; o >>= 1) nv += __shfl_xor_sync(0xffffffffu, nv, o);
            uint64_t t = kEmpty;
            if (nv >= kp) {
                // kEmpty entries sort last, so the kth of all entries is the
                // kth valid one
                const SelectResult sr = warp_select(samp, tot, kp, hist);
                uint64_t mx = 0;
                for (int i = lane; i < tot; i += 32)
                    if (sel_keep(samp[i], sr) && samp[i] > mx) mx = samp[i];
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    const uint64_t y = __shfl_xor_sync(0xffffffffu, mx, o);
                    mx = y > mx ? y : mx;
                }
                t = mx;
            }
            if (lane == 0) {
                thr = t;
                n_cand = best;
            }
        }
        __syncthreads();
        // (2) survivors of the chunk (the current best stays at the front)
        const uint64_t tv = thr;
        for (int base_i = 0; base_i < m; base_i += kThreads) {
            const int i = base_i + tid;
            uint64_t x = kEmpty;
            bool keep = false;
            if (i < m) {
                x = comp(c0 + i);
                keep = x != kEmpty && x <= tv;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            int wpos = 0;
            if (lane == 0 && bal) wpos = atomicAdd(&n_cand, __popc(bal));
            wpos = __shfl_sync(0xffffffffu, wpos, 0);
            const int slot = wpos + __popc(bal & ((1u << lane) - 1u));
            if (keep) cand[slot] = x;
        }
        __syncthreads();
        // (3) keep the k' best
        if (warp == 0) {
            int c = n_cand;
            if (c > kp) {
                const SelectResult sr = warp_select(cand, c, kp, hist);
                uint64_t mx;
                c = warp_pack(cand, c, sr, &mx);
            }
            if (lane == 0) n_cand = c;
        }
        __syncthreads();
        best = n_cand;
    }
    if (best > 0) {
        if (tid == 0) base = atomicAdd(a.out_cnt + b, best);
        __syncthreads();
        uint64_t *o = a.out + (int64_t)b * a.out_cap + base;
        for (int i = tid; i < best; i += kThreads) o[i] = cand[i];
    }
}

}  // namespace

cudaError_t launch_keys_topk(const KeysTopkArgs &a, int parts, cudaStream_t s) {
    if (a.kp > kMaxKp) return cudaErrorInvalidValue;
    dim3 grid(std::max(1, parts), a.B);
    keys_topk_kernel<<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_merge_rerank(const MergeArgs &a, cudaStream_t s) {
    int sort_n = 2;
    while (sort_n < a.kp) sort_n <<= 1;
    size_t sm = (size_t)sort_n * 8 + (size_t)a.stage_cap * 8 + (size_t)a.ldq * 4;
    cudaError_t e = cudaFuncSetAttribute(merge_rerank_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    merge_rerank_kernel<<<a.B, kThreads, sm, s>>>(a, sort_n);
    return cudaGetLastError();
}

}  // namespace vrs
