// k_merge.cu -- per-query final top-k: selection of the k' best first-pass
// candidates, exact FP32 re-rank, sort (ties by the smaller id), output
// padded with id -1 / +inf.
//
// Two front ends feed one finishing stage, one CTA per query:
//  * merge_rerank_kernel: the candidates the distance kernels appended to a
//    per-query list (G*k' composites at most) -- a block radix select of the
//    k' best, staged in shared memory when they fit.
//  * keys_merge_kernel: the query's row of the dense first-pass key matrix,
//    with the minimum of every 128-position chunk of it (both written by the
//    distance pass).  The chunks are split into up to 4 k' groups; the k'
//    smallest group minima are k' distinct keys of the row, so the largest
//    of them, tau, bounds the row's k'-th best key from above, and every key
//    at or below tau lies in a chunk whose minimum is at or below tau.  Only
//    those chunks (about k' of them) are read, their keys at or below tau
//    kept, and the k' best of those selected exactly.  If the candidates
//    overflow the lists, the k' best are selected from the whole row
//    instead.
// Finishing stage: each group of 8 lanes recomputes the exact distance of
// one candidate from the re-rank copy (float32 master, or the stored bf16
// values): L2 in the direct form sum_t (q_t - x_t)^2, IP as q.x -- the form
// the definition uses (Sec. 3, eq. "Brute force similarity search with
// relational predicate"), which avoids the cancellation of the expanded
// ||q||^2 - 2 q.x + ||x||^2 used by the first pass; then a bitonic sort of the
// k' exact composites (in one warp's registers up to 32) and the first k are
// written out.
#include <algorithm>

#include "topk_select.cuh"
#include "vrs_internal.cuh"

namespace vrs {
namespace {

constexpr int kThreads = 256;       // seed_bound_kernel
// merge_rerank_kernel: one block per query; 512 threads halve each query's
// chain of dependent row loads in the re-rank, so the last, partial wave of
// a 1024-query batch (three blocks per SM by registers) ends sooner
constexpr int kRerankThreads = 512;
constexpr int kKeyThreads = 512;    // keys_merge_kernel
constexpr int kChunk = 128;         // positions per chunk minimum
constexpr int kCandChunks = 4096;   // candidate chunk list capacity
constexpr int kGroups = 4096;       // chunk groups for the bound
constexpr int kMinVec = 8;          // chunk minima loaded per thread per round
constexpr int kFallback = 1024;     // widening buffer: k <= 256 plus 4 chunks of 128

// Shared-memory carve: sel[sort_n], list[cap], then the query padded with
// zeros to the master stride (16-byte aligned).
__host__ __device__ inline size_t merge_qs_offset(int sort_n, int cap) {
    return (((size_t)sort_n + (size_t)cap) * 8 + 15) & ~(size_t)15;
}

// In-place exact re-rank of list[0..n): entry i holds a row id in its low
// half and becomes the composite of that row's exact key.  Groups of 8 lanes
// share one entry; n must be the same for every thread of the block.
// U: a lane's 16-byte row loads in flight.  The tensor plans' merge takes 8
// (long rows, hundreds of candidates per query); the dense-key merge keeps 4,
// its code short (it runs once per query, fetched cold after each L2 flush).
template <int U = 4>
__device__ void rerank_list(const MergeArgs &a, uint64_t *list, int n, const float *qs) {
    const int tid = threadIdx.x, lane = tid & 31, T = blockDim.x;
    const int sub = lane & 7, grp = tid >> 3;
    for (int i0 = 0; i0 < n; i0 += T / 8) {
        const int i = i0 + grp;
        float acc = 0.0f;
        int32_t id = 0;
        if (i < n) {
            id = (int32_t)(list[i] & 0xffffffffu);
            const int64_t off = (int64_t)id * a.ld;
#pragma unroll U
            for (int t = sub * 4; t < a.ld; t += 32) {
                float4 x;
                if (a.Xf) {
                    x = __ldg(reinterpret_cast<const float4 *>(a.Xf + off + t));
                } else {
                    const uint2 h = __ldg(reinterpret_cast<const uint2 *>(a.Xb + off + t));
                    x = make_float4(__uint_as_float(h.x << 16), __uint_as_float(h.x & 0xffff0000u),
                                    __uint_as_float(h.y << 16), __uint_as_float(h.y & 0xffff0000u));
                }
                const float4 q = *reinterpret_cast<const float4 *>(qs + t);
                if (a.metric == 0) {
                    const float d0 = q.x - x.x, d1 = q.y - x.y, d2 = q.z - x.z, d3 = q.w - x.w;
                    acc = fmaf(d0, d0, acc);
                    acc = fmaf(d1, d1, acc);
                    acc = fmaf(d2, d2, acc);
                    acc = fmaf(d3, d3, acc);
                } else {
                    acc = fmaf(q.x, x.x, acc);
                    acc = fmaf(q.y, x.y, acc);
                    acc = fmaf(q.z, x.z, acc);
                    acc = fmaf(q.w, x.w, acc);
                }
            }
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        if (i < n && sub == 0) list[i] = make_cand(a.metric == 0 ? acc : -acc, id);
    }
}

// Ascending bitonic sort of v[0..n), n a power of two (one warp's registers
// up to 32).  Every thread of the block calls it.
__device__ void block_sort(uint64_t *v, int n) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, T = blockDim.x;
    if (n <= 32) {
        if (warp == 0) {
            uint64_t x = lane < n ? v[lane] : kEmpty;
#pragma unroll
            for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    const uint64_t y = __shfl_xor_sync(0xffffffffu, x, stride);
                    const bool up = (lane & size) == 0, lower = (lane & stride) == 0;
                    x = (lower == up) ? (x < y ? x : y) : (x < y ? y : x);
                }
            }
            if (lane < n) v[lane] = x;
        }
        __syncthreads();
        return;
    }
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < n / 2; i += T) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const uint64_t x = v[lo], y = v[hi];
                if ((x > y) == up) {
                    v[lo] = y;
                    v[hi] = x;
                }
            }
            __syncthreads();
        }
    }
}

// Block-wide maximum of v[0..n) (kEmpty entries excluded; 0 if none).
__device__ uint64_t block_max(const uint64_t *v, int n, unsigned long long *red) {
    unsigned long long m = 0ull;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (v[i] != kEmpty) m = max(m, (unsigned long long)v[i]);
    if (threadIdx.x == 0) *red = 0ull;
    __syncthreads();
    if (m) atomicMax(red, m);
    __syncthreads();
    const uint64_t r = *red;
    __syncthreads();
    return r;
}

// ||q|| rounded up past the float32 rounding of its sum of squares (qs holds
// the query zero-padded to a.ld).  Every thread calls it; all get the value.
__device__ float query_norm_up(const MergeArgs &a, const float *qs, float *red) {
    const int tid = threadIdx.x;
    if (tid < 32) {
        float ss = 0.0f;
        for (int i = tid; i < a.ld; i += 32) ss = fmaf(qs[i], qs[i], ss);
        for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (tid == 0)
            *red = sqrtf(ss * (1.0f + (float)(a.d + 40) * 5.9604645e-08f)) * 1.0000002f;
    }
    __syncthreads();
    const float r = *red;
    return r;
}

// The certificate parameters with A read from the device when given there.
__device__ __forceinline__ CertArgs cert_of(const MergeArgs &a) {
    CertArgs c = a.cert;
    if (c.A2_dev) c.A = sqrtf(fmaxf(*c.A2_dev, 0.0f)) * 1.0000005f;
    return c;
}

// The certificate of one query (see CertArgs): sel[0..ns) are the exact,
// sorted composites of the candidates, fpk the largest first-pass key among
// them (order-preserving bits), kpq the candidate width, all_rows whether
// every selected row is a candidate.  Returns true when certified; else
// *dup = the k-th exact key rounded up.
__device__ bool certify_with(const CertArgs &c, float rq, int metric, const uint64_t *sel, int ns,
                             int kpq, int kq, uint32_t fpk, float qn, bool all_rows, float *dup) {
    *dup = 0.0f;
    if (kq <= 0 || ns < kpq || all_rows || ns < kq) return true;
    const float D = ordered_to_float((uint32_t)(sel[kq - 1] >> 32));
    *dup = cert_rerank_up(D, qn, c, metric);
    return *dup < ordered_to_float(fpk) - cert_bound(qn, rq, c, metric);
}
__device__ bool certify(const MergeArgs &a, int b, const uint64_t *sel, int ns, int kpq, int kq,
                        uint32_t fpk, float qn, bool all_rows, float *dup) {
    *dup = 0.0f;
    if (kq <= 0 || ns < kpq || all_rows || ns < kq) return true;
    const CertArgs c = cert_of(a);
    return certify_with(c, c.rq ? c.rq[b] : 0.0f, a.metric, sel, ns, kpq, kq, fpk, qn, all_rows,
                        dup);
}

// Lanes per entry for ranking n entries by counting with the 512 threads of
// a block: 8, 4, 2 or 1 (aligned groups of a warp).
__device__ __forceinline__ int rank_lanes(int n) {
    return n <= kKeyThreads / 8 ? 8 : n <= kKeyThreads / 4 ? 4 : n <= kKeyThreads / 2 ? 2 : 1;
}
// Sum of v over the aligned group of L lanes (every lane of the warp calls it).
__device__ __forceinline__ int lane_group_sum(int v, int L) {
    for (int o = 1; o < L; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Ascending bitonic sort of 32 values, one per lane of a warp.
__device__ __forceinline__ uint64_t warp_sort32(uint64_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const uint64_t y = __shfl_xor_sync(0xffffffffu, x, stride);
            const bool up = (lane & size) == 0, lower = (lane & stride) == 0;
            x = (lower == up) ? (x < y ? x : y) : (x < y ? y : x);
        }
    }
    return x;
}

// First kq entries of sel (sorted composites, ns valid) as query b's output
// (id -1 / +inf past them); clears the query's search state.
__device__ void write_out(const MergeArgs &a, int b, const uint64_t *sel, int ns, int kq) {
    const int tid = threadIdx.x, T = blockDim.x;
    for (int i = tid; i < a.k_max; i += T) {
        int64_t id = -1;
        float dist = __int_as_float(0x7f800000);
        if (i < kq && i < ns) {
            const uint64_t c = sel[i];
            id = (int64_t)(c & 0xffffffffu);
            const float key = ordered_to_float((uint32_t)(c >> 32));
            dist = a.metric == 0 ? key : -key;
        }
        a.out_ids[(int64_t)b * a.k_max + i] = id;
        a.out_dist[(int64_t)b * a.k_max + i] = dist;
    }
    if (a.reset_tau && tid == 0) {
        a.reset_tau[b] = kEmpty;
        if (a.cand_cnt) const_cast<int32_t *>(a.cand_cnt)[b] = 0;
    }
}

// Re-rank sel[0..ns) exactly, sort sel[0..sort_n) (entries past ns are
// kEmpty), certify (merge_rerank front end: an uncertified query is flagged
// for a wider pass) and write the first k of query b.  Every thread of the
// block calls it.
__device__ void finish_query(const MergeArgs &a, int b, uint64_t *sel, int ns, int sort_n,
                             const float *qs, int kq, int kpq, bool all_rows) {
    __shared__ unsigned long long red64;
    __shared__ float redf;
    const bool cert = a.rerank && a.cert_flag && !a.dup_only;
    const uint32_t fpk = cert ? (uint32_t)(block_max(sel, ns, &red64) >> 32) : 0u;
    const float qn = (cert || a.dup_only) ? query_norm_up(a, qs, &redf) : 0.0f;
    if (a.rerank) {
        rerank_list<8>(a, sel, ns, qs);
        __syncthreads();
    }
    block_sort(sel, sort_n);
    if (a.dup_only && a.rerank && a.cert_dup && threadIdx.x == 0) {
        float dup = __int_as_float(0x7f800000);
        if (kq > 0 && ns >= kq) {
            const CertArgs c = cert_of(a);
            dup = cert_rerank_up(ordered_to_float((uint32_t)(sel[kq - 1] >> 32)), qn, c, a.metric);
        }
        a.cert_dup[b] = dup;
    }
    if (cert && threadIdx.x == 0) {
        float dup;
        const bool ok = certify(a, b, sel, ns, kpq, kq, fpk, qn, all_rows, &dup);
        a.cert_flag[b] = ok ? 0 : 1;
        if (a.cert_dup) a.cert_dup[b] = dup;
        if (!ok && a.status) atomicMax(a.status, 1);
    }
    if (a.status && a.scan_err && threadIdx.x == 0 && *a.scan_err) atomicMax(a.status, 2);
    write_out(a, b, sel, ns, kq);
}

// Query b's first d values (row stride ldq) into qs, zero-padded to a.ld.
__device__ __forceinline__ void load_query(const MergeArgs &a, int b, float *qs) {
    for (int i = threadIdx.x; i < a.ld; i += blockDim.x)
        qs[i] = i < a.d ? a.Q[(int64_t)b * a.ldq + i] : 0.0f;
}

__global__ void __launch_bounds__(kRerankThreads)
merge_rerank_kernel(MergeArgs a, int sort_n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sel = reinterpret_cast<uint64_t *>(smem_raw);              // [sort_n]
    uint64_t *stg = sel + sort_n;                                         // [stage_cap]
    float *qs = reinterpret_cast<float *>(smem_raw + merge_qs_offset(sort_n, a.stage_cap));
    __shared__ int hist[256];
    __shared__ int scratch[4];
    __shared__ int n_sel, n_valid;

    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
    const int64_t cnt_raw = a.cand_cnt ? (int64_t)a.cand_cnt[b] : a.m;
    const int64_t mq = cnt_raw < a.m ? cnt_raw : a.m;
    const uint64_t *cand = a.cand + (int64_t)b * a.m;
    const int kq = a.k ? a.k[b] : a.k_shared;

    if (tid == 0) {
        n_sel = 0;
        n_valid = 0;
    }
    load_query(a, b, qs);
    // candidates that fit are staged in shared memory: the radix select then
    // makes its passes there instead of over L2
    int nv = 0;
    if (mq <= a.stage_cap) {
#pragma unroll 4
        for (int64_t i = tid; i < mq; i += kRerankThreads) {
            const uint64_t x = cand[i];
            stg[i] = x;
            nv += x != kEmpty;
        }
        cand = stg;
    } else {
        for (int64_t i = tid; i < mq; i += kRerankThreads) nv += cand[i] != kEmpty;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) nv += __shfl_xor_sync(0xffffffffu, nv, o);
    __syncthreads();
    if (lane == 0 && nv) atomicAdd(&n_valid, nv);
    __syncthreads();
    int kpq = a.kp;
    if (a.k && a.kp_factor > 0) {
        kpq = max(kq * a.kp_factor, max(kq + 8, 8 * a.kp_factor));
        kpq = kpq < a.kp ? kpq : a.kp;
    }
    const int want = min(kpq, n_valid);

    SelectResult sr{~0ull, 0ull};   // keeps everything
    if (want < n_valid) sr = block_select(cand, mq, want, hist, scratch);
    for (int64_t i = tid; i < mq; i += kRerankThreads) {
        const uint64_t x = cand[i];
        if (x != kEmpty && sel_keep(x, sr)) sel[atomicAdd(&n_sel, 1)] = x;
    }
    __syncthreads();
    const int ns = n_sel;   // == want
    for (int i = ns + tid; i < sort_n; i += kRerankThreads) sel[i] = kEmpty;
    __syncthreads();
    // (the selected-row count is not read here: block 0 clears it below)
    // sort only the power of two that holds the kept rows and the k written
    // (the entries past ns are kEmpty and sort last)
    int w = 2;
    while (w < ns || w < kq) w <<= 1;
    finish_query(a, b, sel, ns, w < sort_n ? w : sort_n, qs, kq, kpq, false);
    if (a.reset_count && tid == 0 && b == 0) *a.reset_count = 0;
}

// Row id of position pos of query b's key row (c0: the row's first chunk
// in the per-query layout).
__device__ __forceinline__ int32_t key_id(const MergeArgs &a, int64_t c0, int64_t pos) {
    if (a.row_chunk0) return a.row_ids[a.chunk_row[c0 + (pos >> 7)] + (int)(pos & 127)];
    return a.key_ids ? a.key_ids[pos] : (int32_t)pos;
}

// Cold paths of keys_merge_kernel, kept out of line: each step of the
// kernel runs once per query, so its instructions are fetched cold (the
// distance pass's traffic evicts them from L2); out of line, the common
// path's code stays contiguous for the instruction prefetcher.  Every thread
// of the block calls them.

// The bound from G > kKeyThreads group minima (radix select); sets *tau_s
// when at least kp groups hold a key.
__device__ __noinline__ void keys_bound_many(const uint32_t *gmin, int G, int kp, int *hist,
                                             int *scratch, int *n_valid, uint32_t *tau_s) {
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t kInfOrd = float_to_ordered(__int_as_float(0x7f800000));
    auto gcomp = [&](int64_t g) -> uint64_t {
        const uint32_t m = gmin[g];
        return m < kInfOrd ? ((uint64_t)m << 32) | (uint32_t)g : kEmpty;
    };
    int nv = 0;
    for (int g = tid; g < G; g += kKeyThreads) nv += gmin[g] < kInfOrd;
    nv = __reduce_add_sync(0xffffffffu, nv);
    if (lane == 0 && nv) atomicAdd(n_valid, nv);
    __syncthreads();
    if (*n_valid >= kp) {
        uint32_t t = 0;
        const SelectResult sr = block_select_fn(gcomp, G, kp, hist, scratch);
        for (int g = tid; g < G; g += kKeyThreads) {
            const uint64_t x = gcomp(g);
            if (x != kEmpty && sel_keep(x, sr)) t = max(t, (uint32_t)(x >> 32));
        }
        t = __reduce_max_sync(0xffffffffu, t);
        if (tid == 0) *tau_s = 0;
        __syncthreads();
        if (lane == 0) atomicMax(tau_s, t);
        __syncthreads();
    }
}

// The want best of nl > kKeyThreads survivors (radix select), appended to sel.
__device__ __noinline__ void keys_select_many(const uint64_t *lst, int nl, int want, uint64_t *sel,
                                              int *n_sel, int *hist, int *scratch) {
    SelectResult s2{~0ull, 0ull};
    if (want < nl) s2 = block_select(lst, nl, want, hist, scratch);
    for (int i = threadIdx.x; i < nl; i += kKeyThreads)
        if (sel_keep(lst[i], s2)) sel[atomicAdd(n_sel, 1)] = lst[i];
}

// Too many candidates for the lists: the k' best of the whole key row.
__device__ __noinline__ void keys_select_row(const MergeArgs &a, int64_t c0, const float *kb,
                                             int64_t count, uint64_t *sel, int *n_sel, int *n_valid,
                                             int *hist, int *scratch) {
    const int tid = threadIdx.x, lane = tid & 31;
    const float kInf = __int_as_float(0x7f800000);
    auto comp_at = [&](int64_t pos) -> uint64_t {
        const float key = kb[pos];
        return key < kInf ? make_cand(key, key_id(a, c0, pos)) : kEmpty;
    };
    if (tid == 0) *n_valid = 0;
    __syncthreads();
    int nv = 0;
    for (int64_t i = tid; i < count; i += kKeyThreads) nv += kb[i] < kInf;
#pragma unroll
    for (int o = 16; o; o >>= 1) nv += __shfl_xor_sync(0xffffffffu, nv, o);
    if (lane == 0 && nv) atomicAdd(n_valid, nv);
    __syncthreads();
    const int want = min(a.kp, *n_valid);
    SelectResult s2{~0ull, 0ull};
    if (want < *n_valid) s2 = block_select_fn(comp_at, count, want, hist, scratch);
    for (int64_t i = tid; i < count; i += kKeyThreads) {
        const uint64_t x = comp_at(i);
        if (x != kEmpty && sel_keep(x, s2)) sel[atomicAdd(n_sel, 1)] = x;
    }
}

__device__ __noinline__ uint64_t block_max_cold(const uint64_t *v, int n, unsigned long long *red) {
    return block_max(v, n, red);
}
__device__ __noinline__ void block_sort_cold(uint64_t *v, int n) { block_sort(v, n); }

// Scratch of the widening (shared memory of the kernel).
struct WidenSmem {
    uint64_t *fb;        // [kFallback]: top-k, then pending rows
    int32_t *cch;        // [kCandChunks]
    int *n_cch, *n_pend;
    uint32_t *t_ord;
};

// The certificate's widening for query b (see keys_merge_kernel): returns
// with fb[0..kq) the certified top-k.
__device__ __noinline__ void keys_widen(const MergeArgs &a, int b, int64_t c0, const uint64_t *sel,
                                        int kq, int64_t nch, int64_t count, const uint32_t *cm,
                                        const float *kb, uint64_t ckp, float qn, float dup,
                                        const float *qs, WidenSmem w) {
    const int tid = threadIdx.x;
    const float kInf = __int_as_float(0x7f800000);
    const CertArgs cc = cert_of(a);
    const float E = cert_bound(qn, cc.rq ? cc.rq[b] : 0.0f, cc, a.metric);   // thread 0's qn
    if (tid == 0) *w.t_ord = float_to_ordered(dup + E);
    for (int i = tid; i < kq; i += kKeyThreads) w.fb[i] = sel[i];
    __syncthreads();
    for (int64_t cb = 0; cb < nch; cb += kKeyThreads) {
        if (tid == 0) *w.n_cch = 0;
        __syncthreads();
        {
            const int64_t c = cb + tid;
            if (c < nch && cm[c] <= *w.t_ord) w.cch[atomicAdd(w.n_cch, 1)] = (int32_t)c;
        }
        __syncthreads();
        const int nh = *w.n_cch;
        for (int h0 = 0; h0 < nh; h0 += kKeyThreads / kChunk) {
            if (tid == 0) *w.n_pend = 0;
            __syncthreads();
            const int hi = h0 + tid / kChunk;
            if (hi < nh) {
                const int64_t pos = (int64_t)w.cch[hi] * kChunk + (tid % kChunk);
                if (pos < count) {
                    const float key = kb[pos];
                    if (key < kInf && float_to_ordered(key) <= *w.t_ord) {
                        const int32_t id = key_id(a, c0, pos);
                        if (make_cand(key, id) > ckp)
                            w.fb[kq + atomicAdd(w.n_pend, 1)] = (uint32_t)id;
                    }
                }
            }
            __syncthreads();
            const int np = *w.n_pend;
            if (np == 0) continue;
            rerank_list(a, w.fb + kq, np, qs);
            int wd = 2;
            while (wd < kq + np) wd <<= 1;
            for (int i = kq + np + tid; i < wd; i += kKeyThreads) w.fb[i] = kEmpty;
            __syncthreads();
            block_sort(w.fb, wd);
            if (tid == 0) {
                const float D = ordered_to_float((uint32_t)(w.fb[kq - 1] >> 32));
                const uint32_t t2 = float_to_ordered(cert_rerank_up(D, qn, cc, a.metric) + E);
                *w.t_ord = t2 < *w.t_ord ? t2 : *w.t_ord;
            }
            __syncthreads();
        }
    }
}

// One CTA per query over its row of the dense key matrix (see the header).
// cap: list capacity in shared memory (chunk minima, then survivors).  The
// selected-row count is cleared by the last CTA to finish (every CTA reads
// it first).
__global__ void __launch_bounds__(kKeyThreads)
keys_merge_kernel(MergeArgs a, int sort_n, int cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sel = reinterpret_cast<uint64_t *>(smem_raw);   // [sort_n]
    uint64_t *lst = sel + sort_n;                              // [cap]
    float *qs = reinterpret_cast<float *>(smem_raw + merge_qs_offset(sort_n, cap));
    __shared__ __align__(8) int32_t cch[kCandChunks];   // candidate chunks
    __shared__ uint32_t gmin[kGroups];     // group minima (order-preserving keys)
    __shared__ int hist[256];
    __shared__ int scratch[4];
    __shared__ int n_valid, n_cch, n_lst, n_sel, is_last, n_pend;
    __shared__ uint32_t tau_s, t_ord;
    __shared__ bool cert_ok;
    __shared__ float dup_s, redf;
    __shared__ unsigned long long red64, ckp_s;
    __shared__ float qss[kKeyThreads / 32];   // per-warp sums of the query's squares
    __shared__ uint64_t fb[kFallback];   // certificate widening: top-k + pending rows

    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // the query's values are loaded now and stored to shared memory after
    // the bound, so this load overlaps the count and chunk-minimum loads
    constexpr int kQPer = 8;   // ld <= kQPer * kKeyThreads
    float qreg[kQPer];
#pragma unroll
    for (int u = 0; u < kQPer; ++u) {
        const int i = threadIdx.x + u * kKeyThreads;
        qreg[u] = i < a.d ? a.Q[(int64_t)blockIdx.x * a.ldq + i] : 0.0f;
    }
    {
        // ||q||^2 in parts (summed by thread 0 for the certificate; the
        // rounding bound of query_norm_up covers any summation order)
        float ss = 0.0f;
#pragma unroll
        for (int u = 0; u < kQPer; ++u) ss = fmaf(qreg[u], qreg[u], ss);
        for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) qss[warp] = ss;
    }
    // launched as a programmatic dependent of the distance pass: everything
    // it wrote is read after this
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // the query's key row: row b of the matrix, or its own chunks
    int64_t c0 = 0, lim = a.cmin_ld;
    if (a.row_chunk0) {
        c0 = a.row_chunk0[b];
        lim = a.row_chunk0[b + 1] - c0;
    }
    const float *kb = a.row_chunk0 ? a.keys + c0 * kChunk : a.keys + (int64_t)b * a.keys_ld;
    const uint32_t *cm = a.row_chunk0 ? a.chunk_min + c0 : a.chunk_min + (int64_t)b * a.cmin_ld;
    // the first round of chunk minima is loaded together with the count
    // (entries past the count's chunks are masked below)
    uint32_t mv0[kMinVec];
#pragma unroll
    for (int u = 0; u < kMinVec; ++u) {
        const int64_t c = u * kKeyThreads + tid;
        mv0[u] = c < lim ? cm[c] : 0xffffffffu;
    }
    const int64_t count = a.row_chunk0 ? lim * kChunk : *a.key_count;
    // the certificate's inputs, loaded now by the thread that uses them
    const bool cert = a.rerank && a.cert_flag;
    float a2v = 0.0f, rqv = 0.0f;
    if (cert && tid == 0) {
        a2v = a.cert.A2_dev ? *a.cert.A2_dev : 0.0f;
        rqv = a.cert.rq ? a.cert.rq[b] : 0.0f;
    }
    // with the count read from a copy the distance pass left, the original
    // (the filter's accumulator) is cleared for the next query right away
    if (a.reset_count && !a.done && b == 0 && tid == 0) *a.reset_count = 0;
    const int64_t nch = (count + kChunk - 1) / kChunk;
    const float kInf = __int_as_float(0x7f800000);
    const uint32_t kInfOrd = float_to_ordered(kInf);
    const int kq = a.k ? a.k[b] : a.k_shared;
    auto id_at = [&](int64_t pos) -> int32_t { return key_id(a, c0, pos); };
    if (tid == 0) {
        n_valid = 0;
        n_cch = 0;
        n_lst = 0;
        n_sel = 0;
        tau_s = 0xffffffffu;
        ckp_s = 0ull;
    }

    // (1) the bound.  The chunks are split into G = min(nch, 4 k') disjoint
    // groups; the k' smallest group minima are minima of k'
    // distinct chunks, so the k'-th smallest group minimum bounds the row's
    // k'-th best key from above.  One pass over the minima (staged in shared
    // memory when they fit), then a small selection over the G group minima.
    const bool staged = nch <= cap;
    const int gcap = 4 * a.kp < kGroups ? 4 * a.kp : kGroups;
    const int G = (int)(nch < (int64_t)gcap ? nch : (int64_t)gcap);
    for (int g = tid; g < G; g += kKeyThreads) gmin[g] = 0xffffffffu;
    __syncthreads();
    // chunk c belongs to group c % G (a warp's lanes hit different groups);
    // the loads of a round are issued together
    for (int64_t c0 = 0; c0 < nch; c0 += (int64_t)kKeyThreads * kMinVec) {
        uint32_t mv[kMinVec];
#pragma unroll
        for (int u = 0; u < kMinVec; ++u) {
            const int64_t c = c0 + u * kKeyThreads + tid;
            mv[u] = c0 == 0 ? mv0[u] : (c < nch ? cm[c] : 0xffffffffu);
        }
#pragma unroll
        for (int u = 0; u < kMinVec; ++u) {
            const int64_t c = c0 + u * kKeyThreads + tid;
            if (c >= nch) continue;
            const uint32_t m = mv[u];
            if (staged) lst[c] = m < kInfOrd ? ((uint64_t)m << 32) | (uint32_t)c : kEmpty;
            if (m < kInfOrd) atomicMin(&gmin[(int)c % G], m);
        }
    }
    __syncthreads();
    if (nch > a.kp) {
        auto gcomp = [&](int64_t g) -> uint64_t {
            const uint32_t m = gmin[g];
            return m < kInfOrd ? ((uint64_t)m << 32) | (uint32_t)g : kEmpty;
        };
        if (G <= kKeyThreads) {
            // rank by counting: a group of L lanes holds group i's composite
            // and counts the smaller ones; the one of rank k'-1 (if there
            // are k' valid groups) is the bound
            const int L = rank_lanes(G), i = tid / L, sub = tid & (L - 1);
            const uint64_t x = i < G ? gcomp(i) : kEmpty;
            int rank = 0;
            for (int h = sub; h < G; h += L) rank += gcomp(h) < x;
            rank = lane_group_sum(rank, L);
            if (sub == 0 && x != kEmpty && rank == a.kp - 1) tau_s = (uint32_t)(x >> 32);
            __syncthreads();
        } else {
            keys_bound_many(gmin, G, a.kp, hist, scratch, &n_valid, &tau_s);
        }
    }
    const uint32_t tau = tau_s;   // keys at or below it contain the k' best
#pragma unroll
    for (int u = 0; u < kQPer; ++u) {
        const int i = tid + u * kKeyThreads;
        if (i < a.ld) qs[i] = qreg[u];
    }

    // (2) candidate chunks: every chunk whose minimum is at or below tau
    for (int64_t c = tid; c < nch; c += kKeyThreads) {
        const uint32_t m = staged ? (uint32_t)(lst[c] >> 32) : cm[c];
        const bool hit = (staged ? lst[c] != kEmpty : m < kInfOrd) && m <= tau;
        if (hit) {
            const int slot = atomicAdd(&n_cch, 1);
            if (slot < kCandChunks) cch[slot] = (int32_t)c;
        }
    }
    __syncthreads();
    const int ncc = n_cch;

    // (3) one warp per candidate chunk: keys at or below tau, as (key, row
    // id) composites; each chunk's row ids are loaded with its keys
    if (ncc <= kCandChunks) {
        for (int i = warp; i < ncc; i += kKeyThreads / 32) {
            const int64_t p0 = (int64_t)cch[i] * kChunk + lane * 4;
            float4 f = make_float4(kInf, kInf, kInf, kInf);
            int4 iv = make_int4((int)p0, (int)p0 + 1, (int)p0 + 2, (int)p0 + 3);
            if (a.row_chunk0) {
                // a slot's positions past its cell hold +inf (never kept);
                // the ids of the kept keys are looked up below
                f = __ldg(reinterpret_cast<const float4 *>(kb + p0));
            } else if (p0 + 3 < count) {
                f = __ldg(reinterpret_cast<const float4 *>(kb + p0));
                if (a.key_ids) iv = __ldg(reinterpret_cast<const int4 *>(a.key_ids + p0));
            } else {
                if (p0 < count) f.x = kb[p0], iv.x = id_at(p0);
                if (p0 + 1 < count) f.y = kb[p0 + 1], iv.y = id_at(p0 + 1);
                if (p0 + 2 < count) f.z = kb[p0 + 2], iv.z = id_at(p0 + 2);
            }
            const float kv[4] = {f.x, f.y, f.z, f.w};
            int32_t idv[4] = {iv.x, iv.y, iv.z, iv.w};
            unsigned keep = 0;
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (kv[e] < kInf && float_to_ordered(kv[e]) <= tau) keep |= 1u << e;
            if (a.row_chunk0 && keep) {
                const int32_t rb = a.chunk_row[c0 + cch[i]];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if ((keep >> e) & 1u) idv[e] = a.row_ids[rb + lane * 4 + e];
            }
            const int c = __popc(keep);
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            int base = 0;
            if (lane == 31 && incl) base = atomicAdd(&n_lst, incl);
            base = __shfl_sync(0xffffffffu, base, 31);
            int slot = base + incl - c;
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if ((keep >> e) & 1u) {
                    if (slot < cap)
                        lst[slot] = ((uint64_t)float_to_ordered(kv[e]) << 32) | (uint32_t)idv[e];
                    ++slot;
                }
        }
    }
    __syncthreads();
    const int nl = n_lst;

    if (ncc <= kCandChunks && nl <= cap) {
        // the k' best of the survivors
        const int want = min(a.kp, nl);
        if (nl <= kKeyThreads) {
            // rank by counting (composites are unique): survivor i goes to
            // sel[rank] when its rank is below want -- already in key order;
            // the one of rank want-1 is the k'-th first-pass composite
            const int L = rank_lanes(nl), i = tid / L, sub = tid & (L - 1);
            const uint64_t x = i < nl ? lst[i] : kEmpty;
            int rank = 0;
            for (int h = sub; h < nl; h += L) rank += lst[h] < x;
            rank = lane_group_sum(rank, L);
            if (sub == 0 && i < nl && rank < want) {
                sel[rank] = x;
                if (rank == want - 1) ckp_s = x;
            }
            if (tid == 0) n_sel = want;
        } else {
            keys_select_many(lst, nl, want, sel, &n_sel, hist, scratch);
        }
    } else {
        keys_select_row(a, c0, kb, count, sel, &n_sel, &n_valid, hist, scratch);
    }
    __syncthreads();
    const int ns = n_sel;   // == want
    // (the padding is disjoint from the re-ranked entries; the re-rank's
    // barrier orders it before the sort)
    for (int i = ns + tid; i < sort_n; i += kKeyThreads) sel[i] = kEmpty;
    if (!a.rerank) __syncthreads();

    // (4) exact re-rank, sort and the certificate (see CertArgs)
    const bool ckp_known = ncc <= kCandChunks && nl <= cap && nl <= kKeyThreads;
    // k'-th first-pass composite (0 when there are no candidates)
    const uint64_t ckp = !cert ? 0ull : ckp_known ? (uint64_t)ckp_s : block_max_cold(sel, ns, &red64);
    if (a.rerank) {
        rerank_list(a, sel, ns, qs);
        __syncthreads();
    }
    if (sort_n <= 32) {
        // one warp sorts; thread 0 of it certifies before the block meets
        if (warp == 0) {
            const uint64_t x = warp_sort32(lane < sort_n ? sel[lane] : kEmpty);
            if (lane < sort_n) sel[lane] = x;
            __syncwarp();
        }
        if (!cert) __syncthreads();
    } else {
        block_sort_cold(sel, sort_n);
    }
    const uint64_t *res = sel;
    float qn = 0.0f;   // thread 0 only
    if (cert && tid == 0) {
        float ss = 0.0f;
        for (int w = 0; w < kKeyThreads / 32; ++w) ss += qss[w];
        qn = sqrtf(ss * (1.0f + (float)(a.d + 40) * 5.9604645e-08f)) * 1.0000002f;
    }
    if (cert) {
        if (tid == 0) {
            CertArgs c = a.cert;
            if (c.A2_dev) c.A = sqrtf(fmaxf(a2v, 0.0f)) * 1.0000005f;
            float dup;
            cert_ok = certify_with(c, rqv, a.metric, sel, ns, a.kp, kq, (uint32_t)(ckp >> 32), qn,
                                   count <= (int64_t)ns, &dup);
            dup_s = dup;
        }
        __syncthreads();
        if (!cert_ok) {
            // (5) widening: every row whose first-pass key is <= T = D + E may
            // still belong to the top-k.  The rows outside the candidate set
            // (composite above ckp) with a key <= T are re-ranked exactly, 4
            // chunks per round, and merged into the current top-k; T shrinks
            // as the k-th exact key does.
            keys_widen(a, b, c0, sel, kq, nch, count, cm, kb, ckp, qn, dup_s, qs,
                       WidenSmem{fb, cch, &n_cch, &n_pend, &t_ord});
            res = fb;
        }
        if (tid == 0) {
            a.cert_flag[b] = cert_ok ? 0 : 2;
            if (a.cert_dup) a.cert_dup[b] = dup_s;
        }
    }
    write_out(a, b, res, ns, kq);

    // the distance pass finished before this kernel read its output (the
    // launch waits on it), so its error word is final here
    if (a.err_dst && b == 0 && tid == 0) *a.err_dst = *a.err_src;
    // without a count copy, the last CTA to finish clears the selected-row
    // count for the next query
    if (a.reset_count && a.done) {
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            is_last = atomicAdd(a.done, 1) == (int)gridDim.x - 1;
        }
        __syncthreads();
        if (is_last && tid == 0) {
            *a.reset_count = 0;
            *a.done = 0;
        }
    }
}

int sort_width(int kp) {
    int n = 2;
    while (n < kp) n <<= 1;
    return n;
}

// Bound from a sample pass: query b's bound becomes one past the k'-th
// smallest composite of the sample's candidates (every row at or below it
// passes the strict test of the full pass), or kEmpty with fewer than k'
// candidates; the sample's count is cleared for the next query.  With kq,
// query b's width is min(kp, max(kq[b] f, kq[b] + 8, 8 f)), as in the pass.
__global__ void __launch_bounds__(kThreads)
seed_bound_kernel(const uint64_t *__restrict__ cand, int64_t m, int32_t *__restrict__ cnt, int kp,
                  const int32_t *__restrict__ kq, int kp_factor, uint64_t *__restrict__ tau_g) {
    __shared__ int hist[256];
    __shared__ int scratch[4];
    __shared__ unsigned long long kth;
    const int b = blockIdx.x;
    if (kq) {
        const int kk = kq[b];
        kp = min(kp, max(kk * kp_factor, max(kk + 8, 8 * kp_factor)));
    }
    const int64_t nb = min((int64_t)cnt[b], m);
    const uint64_t *v = cand + (int64_t)b * m;
    if (threadIdx.x == 0) kth = 0ull;
    __syncthreads();
    if (nb >= kp) {
        const SelectResult sr = block_select(v, nb, kp, hist, scratch);
        unsigned long long mx = 0ull;
        for (int64_t i = threadIdx.x; i < nb; i += kThreads)
            if (v[i] != kEmpty && sel_keep(v[i], sr)) mx = max(mx, (unsigned long long)v[i]);
        atomicMax(&kth, mx);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        tau_g[b] = nb >= kp ? (uint64_t)kth + 1 : kEmpty;
        cnt[b] = 0;
    }
}

// Row i < m of the staged results goes to row idx[i] of the outputs when
// flag[i] says its query was certified (0 or 2), or always when flag is NULL.
__global__ void scatter_topk_kernel(const int64_t *__restrict__ sid, const float *__restrict__ sd,
                                    const int32_t *__restrict__ idx,
                                    const int32_t *__restrict__ flag, int64_t m, int32_t k_max,
                                    int64_t *__restrict__ oid, float *__restrict__ od) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * k_max) return;
    const int64_t i = t / k_max, j = t % k_max;
    if (flag && flag[i] == 1) return;
    const int64_t o = (int64_t)idx[i] * k_max + j;
    oid[o] = sid[t];
    od[o] = sd[t];
}

}  // namespace

cudaError_t launch_scatter_topk(const int64_t *sid, const float *sd, const int32_t *idx,
                                const int32_t *flag, int64_t m, int32_t k_max, int64_t *oid,
                                float *od, cudaStream_t s) {
    if (!sid || !sd || !idx || !oid || !od || m < 1 || k_max < 1) return cudaErrorInvalidValue;
    const int64_t n = m * k_max;
    scatter_topk_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sid, sd, idx, flag, m, k_max,
                                                                  oid, od);
    return cudaGetLastError();
}

size_t keys_merge_max_smem() {
    static size_t v = 0;   // per process (one GPU model)
    if (v == 0) {
        int dev = 0, optin = 0;
        cudaFuncAttributes fa{};
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, keys_merge_kernel) != cudaSuccess)
            return (size_t)160 << 10;
        v = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    }
    return v;
}

size_t keys_merge_smem(int kp, int cap, int ld) {
    return merge_qs_offset(sort_width(kp), cap) + (size_t)ld * 4;
}

cudaError_t launch_keys_merge(const MergeArgs &a, int cap, cudaStream_t s) {
    if (a.kp > kMaxKp || cap < 1 || a.keys == nullptr ||
        (a.key_count == nullptr && a.row_chunk0 == nullptr) || a.chunk_min == nullptr ||
        (a.row_chunk0 && (!a.chunk_row || !a.row_ids)) || a.ld > 8 * kKeyThreads)
        return cudaErrorInvalidValue;
    const int sort_n = sort_width(a.kp);
    const size_t sm = keys_merge_smem(a.kp, cap, a.ld);
    cudaError_t e = cudaFuncSetAttribute(keys_merge_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    return launch_dependent(keys_merge_kernel, dim3(a.B), dim3(kKeyThreads), sm, s, a, sort_n, cap);
}

cudaError_t launch_merge_rerank(const MergeArgs &a, cudaStream_t s) {
    const int sort_n = sort_width(a.kp);
    const size_t sm = merge_qs_offset(sort_n, a.stage_cap) + (size_t)a.ld * 4;
    cudaError_t e = cudaFuncSetAttribute(merge_rerank_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    merge_rerank_kernel<<<a.B, kRerankThreads, sm, s>>>(a, sort_n);
    return cudaGetLastError();
}

cudaError_t launch_seed_bound(const uint64_t *cand, int64_t m, int32_t *cnt, int B, int kp,
                              const int32_t *kq, int kp_factor, uint64_t *tau_g, cudaStream_t s) {
    if (B < 1 || kp < 1 || m < 1 || (kq && kp_factor < 1)) return cudaErrorInvalidValue;
    seed_bound_kernel<<<B, kThreads, 0, s>>>(cand, m, cnt, kp, kq, kp_factor, tau_g);
    return cudaGetLastError();
}

}  // namespace vrs
