// noalloc.cu -- vrs_query_noalloc: the filtered FP32 top-k query without an
// engine and without any device allocation.
//
// Some callers cannot call cudaMalloc: a host whose own caching allocator
// owns the device's memory pool and forbids allocations beside it, a service
// that fixes its device-memory budget at start-up, or a latency-bound loop
// that must not stall on the driver's allocator.  This entry point runs the
// same kernels as the engine's GEMV plan (predicate -> bitmap, row norms,
// FP32 distance pass with per-CTA top-k', merge + exact re-rank) on
// caller-owned inputs and outputs; everything else it needs lives in one
// file-scope device array of fixed size (kScratchBytes, about 8.4 MB), held
// by every GPU that loads the library until the process exits.
//
// The array's host-side name is only a stand-in for the device object, so
// its device address is obtained once per device with cudaGetSymbolAddress
// (with that device current) and cached.  The first call on each device
// does this set-up; make that first call before any stream capture.
//
// Every call shares the array and it keeps the last call's contents; the
// state that must start cleared (per-query bounds and candidate counts) is
// reset by the call itself.  Calls that overlap on the GPU (different
// streams, or several host threads) race on the array: serialise them.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/vrs.h"
#include "vrs_internal.cuh"

namespace vrs {
vrs_status set_error(vrs_status st, const char *msg);
}

using namespace vrs;

namespace {

// Limits of the no-allocation query (sizes of the scratch regions below).
constexpr int64_t kNaMaxRows = 1 << 20;   // n
constexpr int32_t kNaMaxDim = 1024;       // d (a multiple of 16)
constexpr int32_t kNaMaxBatch = 32;       // queries per call
constexpr int32_t kNaMaxK = 64;           // k
constexpr int32_t kNaKp = 2 * kNaMaxK;    // k' = max(2k, k + 8, 16) candidates re-ranked
constexpr int32_t kNaGrid = 128;          // CTAs per query group of the distance pass

// Scratch layout (byte offsets, each 256-aligned).
constexpr size_t kOffNorms = 0;
constexpr size_t kOffBitmap = kOffNorms + kNaMaxRows * 4;
constexpr size_t kOffTiles = kOffBitmap + kNaMaxRows / 8 + 256;
constexpr size_t kOffQpad = kOffTiles + (kNaMaxRows / kTileRows + 1) * 4 + 256 - 4;
constexpr size_t kOffTau = ((kOffQpad + (size_t)kNaMaxBatch * kNaMaxDim * 4) + 255) / 256 * 256;
constexpr size_t kOffCnt = kOffTau + 256;
constexpr size_t kOffFlag = kOffCnt + 256;   // per-query certificate flags, then max ||x||^2
constexpr size_t kOffCand = kOffFlag + 256;
constexpr size_t kScratchBytes = kOffCand + (size_t)kNaMaxBatch * kNaGrid * kNaKp * 8;
static_assert(kOffBitmap % 256 == 0 && kOffTiles % 256 == 0, "alignment");
static_assert(kOffQpad % 4 == 0 && kOffTau % 256 == 0, "alignment");
static_assert(kNaMaxBatch * 4 + 4 <= 256, "counts and the error word share 256 bytes");
static_assert(kNaMaxBatch * 4 + 4 <= 256, "flags and the norm maximum fit their 256 bytes");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_dev[kMaxDevices] = {};

// Device address of g_scratch on the current device (set up on first use).
vrs_status scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(VRS_ECUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return set_error(VRS_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return set_error(VRS_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
        g_scratch_dev[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_dev[dev];
    return VRS_OK;
}

#define NA_CK(call)                                                          \
    do {                                                                     \
        if ((call) != cudaSuccess) return set_error(VRS_ECUDA, #call " failed"); \
    } while (0)

}  // namespace

extern "C" VRS_API vrs_status vrs_query_noalloc(const float *x, int64_t n, int32_t d,
                                                const int32_t *attrs, int32_t n_cols,
                                                const vrs_pred *pred, const float *q,
                                                int32_t batch, int32_t k, vrs_metric metric,
                                                int64_t *out_ids, float *out_dist,
                                                int32_t *status, void *stream) {
    if (!x || !q || !pred || !out_ids || !out_dist || (n_cols > 0 && !attrs))
        return set_error(VRS_EINVAL, "vrs_query_noalloc: NULL argument");
    if (n < 1 || n > kNaMaxRows)
        return set_error(VRS_EINVAL, "vrs_query_noalloc: n must be in 1..1048576");
    if (d < 16 || d > kNaMaxDim || d % 16)
        return set_error(VRS_EINVAL, "vrs_query_noalloc: d must be a multiple of 16 in 16..1024");
    if (batch < 1 || batch > kNaMaxBatch)
        return set_error(VRS_EINVAL, "vrs_query_noalloc: batch must be in 1..32");
    if (k < 1 || k > kNaMaxK) return set_error(VRS_EINVAL, "vrs_query_noalloc: k must be in 1..64");
    if (metric != VRS_L2 && metric != VRS_IP)
        return set_error(VRS_EINVAL, "vrs_query_noalloc: bad metric");
    if (n_cols < 0 || n_cols > kMaxCols)
        return set_error(VRS_EINVAL, "vrs_query_noalloc: n_cols must be in 0..8");
    if (pred->n_terms < 0 || pred->n_terms > kMaxTerms || (pred->n_terms && !pred->terms))
        return set_error(VRS_EINVAL, "vrs_query_noalloc: bad predicate");
    PredArg p{};
    p.n_terms = pred->n_terms;
    for (int t = 0; t < pred->n_terms; ++t) {
        if (pred->terms[t].col < 0 || pred->terms[t].col >= n_cols)
            return set_error(VRS_EINVAL, "vrs_query_noalloc: predicate column out of range");
        p.col[t] = pred->terms[t].col;
        p.lo[t] = pred->terms[t].lo;
        p.hi[t] = pred->terms[t].hi;
    }
    // the predicate kernel reads attributes 16 bytes at a time, the distance
    // pass reads rows 16 bytes at a time
    if (reinterpret_cast<uintptr_t>(attrs) % 16 || (n_cols > 1 && n % 4))
        return set_error(VRS_EINVAL,
                         "vrs_query_noalloc: attrs must be 16-byte aligned (and n a multiple "
                         "of 4 when n_cols > 1)");
    if (reinterpret_cast<uintptr_t>(x) % 16)
        return set_error(VRS_EINVAL, "vrs_query_noalloc: x must be 16-byte aligned");

    unsigned char *sc = nullptr;
    vrs_status st = scratch_address(&sc);
    if (st != VRS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *norms = reinterpret_cast<float *>(sc + kOffNorms);
    uint32_t *bitmap = reinterpret_cast<uint32_t *>(sc + kOffBitmap);
    int32_t *tiles = reinterpret_cast<int32_t *>(sc + kOffTiles);
    float *qpad = reinterpret_cast<float *>(sc + kOffQpad);
    uint64_t *tau_g = reinterpret_cast<uint64_t *>(sc + kOffTau);
    int32_t *cnt = reinterpret_cast<int32_t *>(sc + kOffCnt);
    // error word of the distance pass, after the counts: each CTA appends at
    // most k' entries per query, so the list cannot overflow; it is cleared
    // here and folded into *status by the merge all the same
    int32_t *err = reinterpret_cast<int32_t *>(sc + kOffCnt + kNaMaxBatch * 4);
    int32_t *flags = reinterpret_cast<int32_t *>(sc + kOffFlag);
    float *xn_max = reinterpret_cast<float *>(sc + kOffFlag + kNaMaxBatch * 4);
    uint64_t *cand = reinterpret_cast<uint64_t *>(sc + kOffCand);

    NA_CK(cudaMemsetAsync(err, 0, 4, s));
    if (status) NA_CK(cudaMemsetAsync(status, 0, 4, s));
    AttrArg aa{};
    for (int c = 0; c < n_cols; ++c) aa.col[c] = attrs + (int64_t)c * n;
    NA_CK(launch_predicate(aa, n, p, bitmap, tiles, s));
    NA_CK(launch_norms_f32(x, n, d, d, norms, s));
    NA_CK(launch_max_f32(norms, n, xn_max, s));
    // resets the per-query bound and candidate count of this call
    NA_CK(launch_prep_queries(q, batch, d, qpad, d, tau_g, cnt, s));

    // the floor keeps a first-pass error band's worth of candidates for small k
    const int kp = std::min(std::max(2 * k, std::max(k + 8, 16)), (int)kNaKp);
    const int G = (int)std::min<int64_t>(kNaGrid, (n + 255) / 256);
    ScanArgs a{};
    a.X = x;
    a.ld = d;
    a.d = d;
    a.xnorm = norms;
    a.ids = nullptr;
    a.bitmap = bitmap;
    a.count_dev = nullptr;
    a.n_rows = n;
    a.Q = qpad;
    a.B = batch;
    a.metric = metric;
    a.kp = kp;
    a.tau_g = tau_g;
    a.out_cnt = cnt;
    a.out = cand;
    a.out_cap = (int64_t)G * kp;
    a.err = err;
    NA_CK(launch_scan_simt(a, G, s));

    MergeArgs m{};
    m.cand = cand;
    m.m = (int64_t)G * kp;
    m.cand_cnt = cnt;
    m.kp = kp;
    m.k = nullptr;
    m.k_shared = k;
    m.k_max = k;
    m.B = batch;
    m.metric = metric;
    m.rerank = 1;
    m.Xf = x;
    m.Xb = nullptr;
    m.ld = d;
    m.d = d;
    m.Q = qpad;
    m.ldq = d;
    m.out_ids = out_ids;
    m.out_dist = out_dist;
    m.stage_cap = (int32_t)std::min<int64_t>(m.m, 4096);
    // the certificate of each query (the FP32 FMA first pass against the
    // exact re-rank; the table's largest norm bounds every row's)
    m.cert_flag = flags;
    m.status = status;
    m.scan_err = err;
    m.cert.A2_dev = xn_max;
    m.cert.Rx = 0.0f;
    m.cert.P = cert_P_ffma(d);
    m.cert.d = d;
    m.cert.rq = nullptr;
    NA_CK(launch_merge_rerank(m, s));
    return VRS_OK;
}
