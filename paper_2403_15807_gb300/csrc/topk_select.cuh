// topk_select.cuh -- exact selection of the kth smallest (key, id) composite.
//
// Candidates are unique uint64 composites (order-preserving float key in the
// high half, row id in the low half), so "the k best" is a set with no ties.
// Selection is an MSD radix select with 8-bit digits: each pass histograms
// the digit of the values that match the prefix chosen so far, and picks the
// bin holding the kth value.  It stops as soon as the chosen bin is taken
// whole, so for distinct float keys it usually ends within the 4 key bytes.
// The result is (prefix, pmask): the selected set is every value v with
// (v & pmask) <= prefix.
#pragma once

#include "vrs_internal.cuh"

namespace vrs {

struct SelectResult {
    uint64_t prefix;
    uint64_t pmask;
};

__device__ __forceinline__ bool sel_keep(uint64_t v, SelectResult r) {
    return (v & r.pmask) <= r.prefix;
}

// Warp-wide: kth smallest (1 <= kth <= m) of v[0..m) in shared or global
// memory.  hist: 256 ints of shared memory owned by this warp.
__device__ inline SelectResult warp_select(const uint64_t *v, int m, int kth, int *hist) {
    const int lane = threadIdx.x & 31;
    uint64_t prefix = 0, pmask = 0;
    int need = kth;
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int i = lane; i < 256; i += 32) hist[i] = 0;
        __syncwarp();
        for (int base = 0; base < m; base += 32) {
            const int i = base + lane;
            int bin = 256;   // no bin
            if (i < m) {
                uint64_t x = v[i];
                if ((x & pmask) == prefix) bin = (int)((x >> shift) & 255);
            }
            // one shared atomic per distinct bin in the warp
            const unsigned grp = __match_any_sync(0xffffffffu, bin);
            if (bin < 256 && lane == __ffs(grp) - 1) atomicAdd(&hist[bin], __popc(grp));
        }
        __syncwarp();
        int h[8], tot = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            h[b] = hist[lane * 8 + b];
            tot += h[b];
        }
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        int excl = incl - tot;
        unsigned ball = __ballot_sync(0xffffffffu, excl < need && need <= incl);
        int src = __ffs(ball) - 1;
        int bin = 0, before = 0, cnt = 0;
        if (lane == src) {
            int c = excl;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                if (c + h[b] >= need) {
                    bin = lane * 8 + b;
                    before = c;
                    cnt = h[b];
                    break;
                }
                c += h[b];
            }
        }
        bin = __shfl_sync(0xffffffffu, bin, src);
        before = __shfl_sync(0xffffffffu, before, src);
        cnt = __shfl_sync(0xffffffffu, cnt, src);
        prefix |= (uint64_t)bin << shift;
        pmask |= 0xFFull << shift;
        need -= before;
        __syncwarp();
        if (cnt == need) break;
    }
    return {prefix, pmask};
}

// Warp-wide in-place compaction of v[0..m) to the values kept by r.
// Returns the kept count; *vmax receives the largest kept value.
__device__ inline int warp_pack(uint64_t *v, int m, SelectResult r, uint64_t *vmax) {
    const int lane = threadIdx.x & 31;
    int out = 0;
    uint64_t mx = 0;
    for (int base = 0; base < m; base += 32) {
        int i = base + lane;
        uint64_t x = i < m ? v[i] : 0;
        bool keep = i < m && sel_keep(x, r);
        unsigned b = __ballot_sync(0xffffffffu, keep);
        __syncwarp();
        if (keep) {
            v[out + __popc(b & ((1u << lane) - 1u))] = x;
            mx = x > mx ? x : mx;
        }
        out += __popc(b);
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        uint64_t y = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = y > mx ? y : mx;
    }
    *vmax = mx;
    return out;
}

// Block-wide version of warp_select over a global array, ignoring kEmpty
// entries.  hist: 256 ints of shared memory; scratch: 4 ints of shared
// memory.  All threads of the block must call it; blockDim.x must be a
// multiple of 32.
template <class Get>
__device__ inline SelectResult block_select_fn(Get get, int64_t m, int kth, int *hist,
                                               int *scratch) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint64_t prefix = 0, pmask = 0;
    int need = kth;
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int64_t base = 0; base < m; base += blockDim.x) {
            const int64_t i = base + tid;
            int bin = 256;
            if (i < m) {
                const uint64_t x = get(i);
                if (x != kEmpty && (x & pmask) == prefix) bin = (int)((x >> shift) & 255);
            }
            const unsigned grp = __match_any_sync(0xffffffffu, bin);
            if (bin < 256 && lane == __ffs(grp) - 1) atomicAdd(&hist[bin], __popc(grp));
        }
        __syncthreads();
        if (warp == 0) {
            int h[8], tot = 0;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                h[b] = hist[lane * 8 + b];
                tot += h[b];
            }
            int incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            int excl = incl - tot;
            if (excl < need && need <= incl) {
                int c = excl;
                for (int b = 0; b < 8; ++b) {
                    if (c + h[b] >= need) {
                        scratch[0] = lane * 8 + b;
                        scratch[1] = c;
                        scratch[2] = h[b];
                        break;
                    }
                    c += h[b];
                }
            }
        }
        __syncthreads();
        int bin = scratch[0], before = scratch[1], cnt = scratch[2];
        prefix |= (uint64_t)bin << shift;
        pmask |= 0xFFull << shift;
        need -= before;
        __syncthreads();
        if (cnt == need) break;
    }
    return {prefix, pmask};
}
__device__ inline SelectResult block_select(const uint64_t *v, int64_t m, int kth, int *hist,
                                            int *scratch) {
    return block_select_fn([v](int64_t i) { return v[i]; }, m, kth, hist, scratch);
}

}  // namespace vrs
