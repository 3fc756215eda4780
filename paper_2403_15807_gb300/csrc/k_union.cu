// k_union.cu -- top-k under a disjunction of conjunctions (richer predicates,
// Table 1 "Any Expression").  The rows a disjunction selects are the union of
// the rows each conjunction selects, so their k best are among the union of
// each conjunction's k best: the query path runs once per conjunction, and
// this kernel merges the lists.  A row that several conjunctions select
// appears in several lists; it is kept once.
//
// One CTA per query: the n_lists x k entries become (key, id) composites
// (key = distance, or -q.x) in shared memory, a bitonic sort orders them, and
// one warp walks the sorted list, skipping ids already taken, until k are out.
#include "vrs_internal.cuh"

namespace vrs {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxEntries = 2048;   // n_lists x k

__global__ void __launch_bounds__(kThreads) union_topk_kernel(UnionArgs a, ListOffsets off,
                                                             int P) {
    __shared__ uint64_t comp[kMaxEntries];
    __shared__ int64_t taken[kMaxK];
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
    const int m = a.n_lists * a.k;
    for (int i = tid; i < P; i += kThreads) {
        uint64_t x = kEmpty;
        if (i < m) {
            const int l = i / a.k, j = i - l * a.k;
            const int64_t o = (int64_t)l * a.list_stride + (int64_t)b * a.k + j;
            const int64_t id = a.ids[o];
            if (id >= 0) {
                const float v = a.dist[o];
                x = make_cand(a.metric == 0 ? v : -v, (int32_t)(id + (l < off.n ? off.v[l] : 0)));
            }
        }
        comp[i] = x;
    }
    __syncthreads();
    // bitonic sort, ascending
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < P / 2; i += kThreads) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const uint64_t x = comp[lo], y = comp[hi];
                if ((x > y) == up) {
                    comp[lo] = y;
                    comp[hi] = x;
                }
            }
            __syncthreads();
        }
    }
    // first k distinct ids in key order (warp 0: each candidate is checked
    // against the ids taken so far, 32 at a time)
    if (tid < 32) {
        int c = 0;
        for (int i = 0; i < P && c < a.k; ++i) {
            const uint64_t x = comp[i];
            if (x == kEmpty) break;
            const int64_t id = (int64_t)(uint32_t)x;
            bool dup = false;
            for (int t = lane; t < c; t += 32) dup = dup || taken[t] == id;
            if (__any_sync(0xffffffffu, dup)) continue;
            if (lane == 0) {
                taken[c] = id;
                const float key = ordered_to_float((uint32_t)(x >> 32));
                a.out_ids[(int64_t)b * a.k + c] = id;
                a.out_dist[(int64_t)b * a.k + c] = a.metric == 0 ? key : -key;
            }
            ++c;
            __syncwarp();
        }
        for (int t = c + lane; t < a.k; t += 32) {
            a.out_ids[(int64_t)b * a.k + t] = -1;
            a.out_dist[(int64_t)b * a.k + t] = __int_as_float(0x7f800000);
        }
    }
}

}  // namespace

int union_max_entries() { return kMaxEntries; }

cudaError_t launch_union_topk(const UnionArgs &a, cudaStream_t s, const ListOffsets *off) {
    const int m = a.n_lists * a.k;
    if (a.B < 1 || a.n_lists < 1 || a.k < 1 || a.k > kMaxK || m > kMaxEntries || !a.ids ||
        !a.dist || !a.out_ids || !a.out_dist || (off && (off->n < 0 || off->n > kMaxLists)))
        return cudaErrorInvalidValue;
    int P = 2;
    while (P < m) P <<= 1;
    ListOffsets o{};
    if (off) o = *off;
    union_topk_kernel<<<a.B, kThreads, 0, s>>>(a, o, P);
    return cudaGetLastError();
}

}  // namespace vrs
