// engine.cu -- the C ABI (include/vrs.h): argument checking, device
// storage of the table R (Sec. 3: a column store of one vector column and
// int32 relational columns), the query pipeline and the plan rule.
//
// Query pipeline (Sec. 3.2 predicate pushdown, then Sec. 3.1 scan):
//   predicate -> bitmap + tile counts -> tile offsets -> ascending ids
//   -> (exact count read back; plan chosen) -> distance pass with fused
//   per-CTA top-k' -> merge + exact FP32 re-rank -> top-k.
#include <cuda_runtime.h>

#include <dlfcn.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/vrs.h"
#include "vrs_internal.cuh"

namespace vrs {
size_t scan_simt_smem(int QB, int ld, int kp);
}

using namespace vrs;

namespace {

constexpr int64_t kSampleRows = 16384;

thread_local std::string g_err;

vrs_status fail(vrs_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? VRS_ENOMEM : VRS_ECUDA,         \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                        \
    } while (0)

#define TRY(expr)                          \
    do {                                   \
        vrs_status s_ = (expr);            \
        if (s_ != VRS_OK) return s_;       \
    } while (0)

// Incremented whenever any workspace buffer is (re)allocated: a captured
// CUDA graph is only replayed while the epoch it was captured at holds.
uint64_t g_ws_epoch = 1;

bool fault_alloc() {
    const char *f = getenv("VRS_FAULT");
    return f && strcmp(f, "alloc") == 0;
}

// A growable device buffer.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    vrs_status ensure(size_t need) {
        if (need <= bytes && p) return VRS_OK;
        if (fault_alloc()) return fail(VRS_ENOMEM, "allocation of %zu bytes failed (injected)", need);
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        size_t want = std::max<size_t>(need, 256);
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return fail(VRS_ENOMEM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
        }
        bytes = want;
        ++g_ws_epoch;
        return VRS_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

int32_t round_up(int32_t x, int32_t m) { return (x + m - 1) / m * m; }

}  // namespace

struct vrs_engine {
    int device = 0;
    int n_sm = 152;
    int64_t n = 0;
    int32_t d = 0, ld = 0;
    bool has[3] = {false, false, false};   // resident encodings by vrs_dtype
    bool bf16_is_master = false;          // stored values are the bf16 input
    DevBuf x32, xb, x8, s8, norms;
    DevBuf xp;                            // bf16 pair copy of the float32 rows (VRS_OPT_PAIR_COPY)
    bool pair_copy = true;                // VRS_OPT_PAIR_COPY
    bool wait_test = false;               // VRS_OPT_WAIT_TEST (one-shot)
    bool cert_sample = true;              // VRS_OPT_CERT_SAMPLE
    DevBuf attr[kMaxCols];
    bool attr_loaded[kMaxCols] = {};
    // strided host sample of each attribute column (rows i*n/S), used to
    // estimate a predicate's selectivity without a device round trip
    std::vector<int32_t> attr_sample[kMaxCols];
    // workspace
    DevBuf bitmap, tile_counts, tile_offsets, count, ids, qin, qpad, cand, oid, odist, staging;
    DevBuf tau_g, cand_cnt;   // per-query global bound and candidate count
    DevBuf count_q;           // selected-row count of the query path (zeroed by the merge)
    DevBuf cmin;              // dense-key mode: per-chunk key minima [batch x ceil(n/128)]
    DevBuf qenc, qnorm, qscale, heap_g, err;   // tensor path
    int32_t *h_err = nullptr;  // pinned
    int64_t *h_count = nullptr;   // pinned
    int plan_forced = VRS_PLAN_AUTO;
    int last_plan = VRS_PLAN_GEMV;
    int kprime_factor = 0;
    int rerank = 1;
    int grid_ctas = 0;
    bool fused_gemv = false;  // VRS_OPT_FUSED_SCAN
    bool batched = true;      // VRS_OPT_BATCHED
    bool use_graph = true;    // VRS_OPT_GRAPH
    bool tma = true;          // VRS_OPT_TMA
    bool dense_keys = true;   // VRS_OPT_DENSE_KEYS
    int64_t select_cap = 0;   // VRS_OPT_SELECT_CAP (0: derived)
    bool staged_scan = false; // VRS_OPT_STAGED_SCAN
    bool tensor_gemv = true;  // VRS_OPT_TENSOR_GEMV
    bool seed_bound = true;   // VRS_OPT_SEED_BOUND
    cudaStream_t own = nullptr;   // host-buffer queries without a stream run here
    DevBuf pred_dev;          // device copy of the query's predicate
    // what pred_dev holds (uploaded on pred_stream), and the pinned ring the
    // uploads go through (a slot is reused once its copy has completed)
    static constexpr int kPredRing = 16;
    PredArg pred_up{};
    bool pred_up_valid = false;
    cudaStream_t pred_stream = nullptr;
    PredArg *pred_pin = nullptr;
    cudaEvent_t pred_ev[kPredRing] = {};
    bool pred_ev_used[kPredRing] = {};
    int pred_slot = 0;
    // last selectivity estimate (the attribute samples change only on load)
    PredArg sel_p{};
    double sel_v = 0.0;
    bool sel_valid = false;
    DevBuf smp_ids, smp_count, smp_cand, smp_cnt;   // sample pass of the tensor plans
    DevBuf xn_max;            // max ||x||^2 (range search margin), valid when xn_max_valid
    bool xn_max_valid = false;
    DevBuf rcount, roff, rids, rdist;   // range search: counts, offsets, staged results
    // vector join: the query relation (rows, attributes), its selection, the
    // gathered queries and staged results
    DevBuf jq, jqa, jbm, jtc, jto, jcnt, jqids, jgq, joid, jodist;
    DevBuf uids, udist;       // disjunctions: one top-k list per conjunction
    int64_t *h_rcount = nullptr;        // pinned [65]
    // graphs of the shared-predicate pipeline, by shape key (oldest evicted)
    struct GraphEntry {
        std::string key;
        cudaGraphExec_t exec = nullptr;
        std::vector<cudaEvent_t> evs;
        struct M { int stage; int a, b; };
        std::vector<M> marks;   // indexes into evs
    };
    std::vector<GraphEntry> graphs;
    std::string pending_key;    // eager run seen once; captured on the next one
    bool capturing = false;
    GraphEntry *cap = nullptr;
    DevBuf keys;              // first-pass key matrix of the dense-key GEMV
    // learned plan model (vrs_planner_load)
    bool planner = false;
    float pl_fmean[6], pl_fstd[6], pl_omean = 0.0f, pl_ostd = 1.0f;
    std::vector<float> pl_params;   // 4803, rounded to bf16 at load
    DevBuf qrange, kdev;      // batched launch: per-query ranges and k
    std::vector<int32_t> h_qrange;
    // CUDA graph of the batched kernel sequence, keyed by its shape
    cudaGraphExec_t graph = nullptr;
    std::string graph_key;
    // autotuned CTAs per query tile, keyed by shape
    std::vector<std::pair<std::string, int>> tuned;
    // profiling (VRS_OPT_PROFILE)
    bool profile = false;
    bool profiled_last = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    struct Mark { int stage; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    int32_t launches = 0;
    int64_t last_count = 0;
    // exactness certificate: load-time statistics (max ||x|| of the re-rank
    // copy; max ||x - x_enc|| of each encoding), the per-query flags and
    // k-th exact keys of the current merge, the query residuals of the
    // tensor path, and counters of how queries were certified
    float cert_A = 0.0f;
    float cert_Rx[3] = {0.0f, 0.0f, 0.0f};
    DevBuf stats, cflag, cdup, qres;
    int32_t *cur_cflag = nullptr;   // where the next merge writes its flags
    float *cur_cdup = nullptr;
    bool rerank_merge = false;      // the last merge may leave uncertified queries
    int first_pass = 0;             // kernel family of the current first pass (CertKind)
    vrs_dtype first_src = VRS_F32;  // the encoding it reads
    const float *first_rq = nullptr;   // its per-query residuals (tensor plans)
    int fb_kp = 0;                  // > 0: candidate width of a widened pass
    const float *fb_seed = nullptr; // widened pass: the k-th exact keys its bound starts from
    // fallback chain buffers: query subset, gathered rows, staged results
    DevBuf fb_idx, fb_q, fb_dup, fb_k, fb_oid, fb_odist, fb_flag, fb_dup2;
    int64_t cert_count[4] = {0, 0, 0, 0};   // first pass / in-merge widening / wider pass / exact GEMV
    // flags of the last self-certified pass, counted when asked for (or
    // before the next pass overwrites them) so the pass stays asynchronous
    const int32_t *cert_lazy = nullptr;
    int32_t cert_lazy_n = 0;
    cudaStream_t cert_lazy_s = nullptr;
    // a host-buffer query on the captured GEMV form: the query upload, the
    // result downloads and the error-word read go into the same graph
    const float *io_q_host = nullptr;
    int64_t *io_ids_host = nullptr;
    float *io_dist_host = nullptr;
    size_t io_q_bytes = 0, io_out_n = 0;
    bool io_out_done = false;
    // device addresses of those page-locked host buffers (the host memory is
    // in the device's address space): with VRS_OPT_ZERO_COPY the captured
    // GEMV form reads the queries and writes the results there directly
    const float *io_q_dev = nullptr;
    int64_t *io_ids_dev = nullptr;
    float *io_dist_dev = nullptr;
    bool zero_copy = true;   // VRS_OPT_ZERO_COPY
    int32_t *h_err_dev = nullptr;   // device address of h_err
    bool err_to_host = false;       // the dense-key merge writes the error word to h_err
    // two-column grid of the cell plan (vrs_build_grid): bins of the two
    // columns (bin b holds values [edge[b], edge[b+1])), the clustered copy
    // and, on the host, each cell's rows and chunks with their summed-area
    // table (chunks of any rectangle of cells in O(1))
    struct CellGrid {
        bool valid = false;
        int col[2] = {-1, -1};
        int nb[2] = {0, 0};
        int32_t row_bytes = 0;           // clustered row stride
        std::vector<int64_t> edge[2];
        std::vector<int64_t> off;        // [cells + 1]
        std::vector<int32_t> nch;        // [cells]
        std::vector<int64_t> sat;        // [(nb0 + 1) x (nb1 + 1)]
        DevBuf xg, ng, g0, g1, ids, off_d, nch_d;
        CUtensorMap tmX;
        void release() {
            valid = false;
            for (DevBuf *b : {&xg, &ng, &g0, &g1, &ids, &off_d, &nch_d}) b->release();
        }
    } grid;
    bool cell_plan = true;   // VRS_OPT_CELL_PLAN
    // page-locked staging of per-call uploads (two slots, each reused once
    // the copies last issued from it completed), so those copies do not
    // wait for the stream's earlier work
    struct PinSlot {
        void *p = nullptr;
        size_t bytes = 0;
        cudaEvent_t ev = nullptr;
        bool used = false;
    } pin[2];
    int pin_next = 0;
    // per-batch buffers of the cell plan
    DevBuf c_rect, c_qchunk0, c_entry0, c_cursor, c_entries, c_items, c_qrange, c_keys, c_cmin, c_crow;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Stage timing: when profiling, each stage is bracketed by two events
// recorded on the query's stream.
// Tracing: every entry point that runs work is an NVTX range, and each
// stage's end an NVTX mark (no cost unless a profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
const char *const kStageName[VRS_N_STAGES] = {"vrs prepare", "vrs predicate", "vrs offsets",
                                              "vrs compact", "vrs distance", "vrs merge"};

struct StageTimer {
    vrs_engine *e;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    StageTimer(vrs_engine *e_, cudaStream_t s_) : e(e_), s(s_) {}
    int ia = -1;
    cudaEvent_t take() {
        if (e->capturing) {   // events that live with the captured graph
            cudaEvent_t ev;
            if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
            e->cap->evs.push_back(ev);
            return ev;
        }
        if (e->ev_used == e->ev_pool.size()) {
            cudaEvent_t ev;
            if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
            e->ev_pool.push_back(ev);
        }
        return e->ev_pool[e->ev_used++];
    }
    void record(cudaEvent_t ev) {
        if (e->capturing) cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
        else cudaEventRecord(ev, s);
    }
    void begin() {
        if (!e->profile) return;
        a = take();
        if (a) {
            record(a);
            ia = e->capturing ? (int)e->cap->evs.size() - 1 : -1;
        }
    }
    void end(int stage) {
        if (stage >= 0 && stage < VRS_N_STAGES) nvtxMarkA(kStageName[stage]);
        if (!e->profile || !a) return;
        cudaEvent_t b = take();
        if (!b) return;
        record(b);
        if (e->capturing) e->cap->marks.push_back({stage, ia, (int)e->cap->evs.size() - 1});
        else e->marks.push_back({stage, a, b});
        a = nullptr;
    }
};

vrs_status check_pred(const vrs_engine *e, const vrs_pred *p, PredArg *out) {
    if (!p) return fail(VRS_EINVAL, "predicate pointer is NULL");
    if (p->n_terms < 0 || p->n_terms > kMaxTerms)
        return fail(VRS_EINVAL, "predicate has %d terms (0..%d allowed)", p->n_terms, kMaxTerms);
    if (p->n_terms > 0 && !p->terms) return fail(VRS_EINVAL, "predicate terms pointer is NULL");
    memset(out, 0, sizeof *out);
    out->n_terms = p->n_terms;
    for (int t = 0; t < p->n_terms; ++t) {
        const vrs_range &r = p->terms[t];
        if (r.col < 0 || r.col >= kMaxCols)
            return fail(VRS_EINVAL, "predicate term %d: column %d out of range", t, r.col);
        if (!e->attr_loaded[r.col])
            return fail(VRS_ESTATE, "predicate term %d: column %d not loaded", t, r.col);
        out->col[t] = r.col;
        out->lo[t] = r.lo;
        out->hi[t] = r.hi;
    }
    return VRS_OK;
}

AttrArg attr_arg(const vrs_engine *e) {
    AttrArg a;
    for (int c = 0; c < kMaxCols; ++c) a.col[c] = e->attr[c].as<const int32_t>();
    return a;
}

int64_t n_tiles(int64_t n) { return (n + kTileRows - 1) / kTileRows; }

// Selectivity estimate of a predicate from the attribute samples.
double estimate_selectivity(vrs_engine *e, const PredArg &p) {
    if (p.n_terms == 0) return 1.0;
    if (e->sel_valid && std::memcmp(&e->sel_p, &p, sizeof(PredArg)) == 0) return e->sel_v;
    const size_t S = e->attr_sample[p.col[0]].size();
    if (S == 0) return 1.0;
    size_t hit = 0;
    for (size_t j = 0; j < S; ++j) {
        bool ok = true;
        for (int t = 0; t < p.n_terms && ok; ++t) {
            int32_t v = e->attr_sample[p.col[t]][j];
            ok = p.lo[t] <= v && v < p.hi[t];
        }
        hit += ok;
    }
    e->sel_p = p;
    e->sel_v = (double)hit / (double)S;
    e->sel_valid = true;
    return e->sel_v;
}

// Make pred_dev hold p for work enqueued on s: nothing to do when it already
// does (uploaded on the same stream), else an asynchronous copy from a slot
// of the pinned ring.
vrs_status upload_pred(vrs_engine *e, const PredArg &p, cudaStream_t s) {
    if (e->pred_up_valid && e->pred_stream == s && std::memcmp(&e->pred_up, &p, sizeof(PredArg)) == 0)
        return VRS_OK;
    TRY(e->pred_dev.ensure(sizeof(PredArg)));
    if (!e->pred_pin) {
        void *h = nullptr;
        CK(cudaMallocHost(&h, sizeof(PredArg) * vrs_engine::kPredRing));
        e->pred_pin = static_cast<PredArg *>(h);
        for (auto &ev : e->pred_ev) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    const int slot = e->pred_slot;
    e->pred_slot = (slot + 1) % vrs_engine::kPredRing;
    if (e->pred_ev_used[slot]) CK(cudaEventSynchronize(e->pred_ev[slot]));
    e->pred_pin[slot] = p;
    CK(cudaMemcpyAsync(e->pred_dev.p, &e->pred_pin[slot], sizeof(PredArg), cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(e->pred_ev[slot], s));
    e->pred_ev_used[slot] = true;
    e->pred_up = p;
    e->pred_stream = s;
    e->pred_up_valid = true;
    return VRS_OK;
}

// predicate -> bitmap, tile counts, offsets, device total
vrs_status run_filter(vrs_engine *e, const PredArg &p, cudaStream_t s) {
    const int64_t nt = n_tiles(e->n);
    TRY(e->bitmap.ensure((size_t)((e->n + 31) / 32) * 4 + 16));
    TRY(e->tile_counts.ensure((size_t)nt * 4));
    TRY(e->tile_offsets.ensure((size_t)nt * 8));
    TRY(e->count.ensure(64));
    StageTimer t(e, s);
    t.begin();
    CK(launch_predicate(attr_arg(e), e->n, p, e->bitmap.as<uint32_t>(), e->tile_counts.as<int32_t>(), s));
    t.end(VRS_STAGE_PREDICATE);
    t.begin();
    CK(launch_tile_scan(e->tile_counts.as<int32_t>(), nt, e->tile_offsets.as<int64_t>(),
                        e->count.as<int64_t>(), s));
    t.end(VRS_STAGE_OFFSETS);
    e->launches += 2;
    return VRS_OK;
}

vrs_status run_compact(vrs_engine *e, cudaStream_t s) {
    TRY(e->ids.ensure((size_t)e->n * 4));
    StageTimer t(e, s);
    t.begin();
    CK(launch_compact(e->bitmap.as<uint32_t>(), e->n, e->tile_offsets.as<int64_t>(),
                      e->ids.as<int32_t>(), s));
    t.end(VRS_STAGE_COMPACT);
    e->launches += 1;
    return VRS_OK;
}

// predicate -> unordered ids + count in one kernel (plans that only need
// the set of qualifying rows); the count is zeroed by the previous merge
vrs_status run_filter_ids(vrs_engine *e, const PredArg &p, cudaStream_t s) {
    TRY(e->ids.ensure((size_t)e->n * 4));
    const size_t before = e->count_q.bytes;
    TRY(e->count_q.ensure(64));
    if (e->count_q.bytes != before) CK(cudaMemsetAsync(e->count_q.p, 0, e->count_q.bytes, s));
    StageTimer t(e, s);
    t.begin();
    CK(launch_predicate_ids(attr_arg(e), e->n, p, nullptr, e->ids.as<int32_t>(),
                            e->count_q.as<int64_t>(), e->n_sm, s));
    t.end(VRS_STAGE_PREDICATE);
    e->launches += 1;
    return VRS_OK;
}

vrs_status read_count(vrs_engine *e, cudaStream_t s, int64_t *out) {
    CK(cudaMemcpyAsync(e->h_count, e->count.p, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *out = *e->h_count;
    return VRS_OK;
}

// Fixed plan rule.  From the paper's takeaways: a per-tuple scan for small
// batches, the batched tensor formulation for large ones (Sec. 5.1/5.2), and
// the decision driven by selectivity, dimension and batch (Sec. 5.3).
// ---------------------------------------------------------------------------
// Learned plan model: host evaluation of the 6-64-64-3 network in its bf16
// inference form (weights, inputs and activations rounded to bf16, float32
// accumulation) -- the same arithmetic as the device kernel.
// ---------------------------------------------------------------------------
constexpr int kPlIn = 6, kPlH = 64, kPlOut = 3, kPlNP = 4803;

float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

void planner_predict(const vrs_engine *e, const float *feat, float *y) {
    const float *P = e->pl_params.data();
    const float *W1 = P, *b1 = W1 + kPlH * kPlIn, *W2 = b1 + kPlH, *b2 = W2 + kPlH * kPlH,
                *W3 = b2 + kPlH, *b3 = W3 + kPlOut * kPlH;
    float x[kPlIn], h1[kPlH], h2[kPlH];
    for (int c = 0; c < kPlIn; ++c) x[c] = bf16r((feat[c] - e->pl_fmean[c]) / e->pl_fstd[c]);
    for (int r = 0; r < kPlH; ++r) {
        float s = b1[r];
        for (int c = 0; c < kPlIn; ++c) s = fmaf(W1[r * kPlIn + c], x[c], s);
        h1[r] = bf16r(s > 0.0f ? s : 0.0f);
    }
    for (int r = 0; r < kPlH; ++r) {
        float s = b2[r];
        for (int c = 0; c < kPlH; ++c) s = fmaf(W2[r * kPlH + c], h1[c], s);
        h2[r] = bf16r(s > 0.0f ? s : 0.0f);
    }
    for (int o = 0; o < kPlOut; ++o) {
        float s = b3[o];
        for (int c = 0; c < kPlH; ++c) s = fmaf(W3[o * kPlH + c], h2[c], s);
        y[o] = s;
    }
}

uint64_t fnv1a(const unsigned char *p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

// Plan of smallest predicted latency among those the dtype supports.
int planner_choice(const vrs_engine *e, int32_t batch, double s_est, int32_t k,
                   vrs_dtype compute) {
    const double bpe = compute == VRS_F32 ? 4.0 : compute == VRS_BF16 ? 2.0 : 1.0;
    const float feat[kPlIn] = {(float)std::log((double)e->n), (float)std::log((double)e->d),
                               (float)std::log((double)batch),
                               (float)std::log(std::max(s_est, 1e-6)),
                               (float)std::log((double)std::max(k, 1)), (float)bpe};
    float y[kPlOut];
    planner_predict(e, feat, y);
    const bool ok[3] = {compute != VRS_FP8E4M3, compute != VRS_F32, compute != VRS_F32};
    int best = -1;
    for (int p = 0; p < 3; ++p)
        if (ok[p] && (best < 0 || y[p] < y[best])) best = p;
    return best;
}

//  * FP32 compute runs the per-tuple scan on CUDA cores (GEMV plan);
//  * reduced precision runs the tensor formulation: predicate first with the
//    qualifying rows gathered (COMPACT_GEMM) when few rows qualify, the
//    dense product with the predicate applied to the scores (MASK_GEMM)
//    when at least half of the rows qualify and gathering saves little.
// Reduced precision: the dense scan wins once the gathered rows cost more
// than scanning all rows with the mask; measured at 1M x 960, 1024 queries,
// the crossover is near 30 % (BF16) and 20 % (E4M3).
int fixed_rule(const vrs_engine *e, int32_t batch, double s_est, vrs_dtype compute) {
    (void)e;
    (void)batch;
    if (compute == VRS_F32) return VRS_PLAN_GEMV;
    return s_est >= (compute == VRS_FP8E4M3 ? 0.2 : 0.3) ? VRS_PLAN_MASK_GEMM
                                                         : VRS_PLAN_COMPACT_GEMM;
}

// Device error word (set by bounded waits that gave up); checked whenever
// the host synchronises with the query's stream.
vrs_status check_device_error(vrs_engine *e, cudaStream_t s) {
    CK(cudaMemcpyAsync(e->h_err, e->err.p, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (*e->h_err) {
        const int32_t code = *e->h_err;
        CK(cudaMemsetAsync(e->err.p, 0, 4, s));
        // the failed query may have left its per-query state set: clear it, so
        // that the next query starts as after a completed one
        if (e->count_q.p) CK(cudaMemsetAsync(e->count_q.p, 0, e->count_q.bytes, s));
        if (e->tau_g.p) CK(cudaMemsetAsync(e->tau_g.p, 0xFF, e->tau_g.bytes, s));
        if (e->cand_cnt.p) CK(cudaMemsetAsync(e->cand_cnt.p, 0, e->cand_cnt.bytes, s));
        if (e->smp_cnt.p) CK(cudaMemsetAsync(e->smp_cnt.p, 0, e->smp_cnt.bytes, s));
        CK(cudaStreamSynchronize(s));
        if (code == 2)
            return fail(VRS_EINTERNAL, "a candidate list overflowed its capacity; results are invalid");
        return fail(VRS_ETIMEOUT, "a device-side wait timed out; results are invalid");
    }
    return VRS_OK;
}

// first-pass error grows from FP32 (2k) to BF16 (8 significant bits: 4k)
// to E4M3 (4 significant bits: 16k)
int kprime_factor(const vrs_engine *e, vrs_dtype compute) {
    return e->kprime_factor > 0 ? e->kprime_factor
                                : (compute == VRS_F32 ? 2 : compute == VRS_BF16 ? 4 : 16);
}

// k' = max(f k, k + 8, 8 f): the floor 8 f keeps a first-pass error band's
// worth of candidates for small k
int default_kprime(const vrs_engine *e, int32_t k, vrs_dtype compute) {
    const int f = kprime_factor(e, compute);
    int kp = std::max(k * f, std::max(k + 8, 8 * f));
    return std::min(kp, kMaxKp);
}

// First-pass kernel families (their product error factors, CertArgs.P).
enum CertKind { kCertFFMA = 0, kCertTF32x3 = 1, kCertBF16x3 = 2, kCertBF16 = 3, kCertE4M3 = 4 };

// Certificate parameters of the current first pass (kind, the encoding it
// read, the queries' residuals).
CertArgs cert_args(const vrs_engine *e) {
    CertArgs c{};
    c.A = e->cert_A;
    c.Rx = e->cert_Rx[e->first_src];
    c.d = e->d;
    c.rq = e->first_rq;
    switch (e->first_pass) {
        case kCertTF32x3: c.P = cert_P_tf32x3(e->d); break;
        case kCertBF16x3: c.P = cert_P_bf16x3(e->d); break;
        case kCertBF16: c.P = cert_P_bf16(e->d); break;
        case kCertE4M3: c.P = cert_P_e4m3(e->d); break;
        default: c.P = cert_P_ffma(e->d); break;
    }
    return c;
}

void set_first_pass(vrs_engine *e, int kind, vrs_dtype src, const float *rq) {
    e->first_pass = kind;
    e->first_src = src;
    e->first_rq = rq;
}

vrs_status run_merge(vrs_engine *e, const float *q_dev, int32_t ldq, uint64_t *tau_g,
                     int32_t *cand_cnt, int64_t out_cap, int32_t batch, int kp,
                     const int32_t *k_dev, int32_t k_shared, int32_t k_max, vrs_metric metric,
                     int64_t *oid, float *odist, cudaStream_t s) {
    MergeArgs m{};
    m.cand = e->cand.as<const uint64_t>();
    m.m = out_cap;
    m.cand_cnt = cand_cnt;
    m.kp = kp;
    m.k = k_dev;
    m.k_shared = k_shared;
    m.k_max = k_max;
    m.B = batch;
    m.metric = metric;
    m.rerank = e->rerank;
    m.Xf = e->has[VRS_F32] ? e->x32.as<const float>() : nullptr;
    m.Xb = e->has[VRS_F32] ? nullptr : e->xb.as<const uint16_t>();
    m.ld = e->ld;
    m.d = e->d;
    m.Q = q_dev;
    m.ldq = ldq;
    m.out_ids = oid;
    m.out_dist = odist;
    m.reset_tau = tau_g;
    m.reset_count = e->count_q.p ? e->count_q.as<int64_t>() : nullptr;
    // wide lists (the certifying pass's k') skip the shared-memory staging of
    // the candidates: half the block's shared memory, twice the blocks per SM
    // for the re-rank, which then dominates
    m.stage_cap = kp >= 2048 ? 0 : (int32_t)std::min<int64_t>(out_cap, 4096);
    m.cert = cert_args(e);
    m.cert_flag = e->cur_cflag;
    m.cert_dup = e->cur_cdup;
    e->rerank_merge = true;
    StageTimer t(e, s);
    t.begin();
    CK(launch_merge_rerank(m, s));
    t.end(VRS_STAGE_MERGE);
    e->launches += 1;
    return VRS_OK;
}

// Selected rows per CTA of the full pass from which the sample pass below
// is used (BF16 MASK_GEMM; E4M3 on either plan).
constexpr int64_t kSeedMinRows = 8192;
constexpr int64_t kSeedMinRowsE4M3 = 2048;
// Buffers of the sample pass (the per-query counts start at zero and are
// cleared again by the bound kernel).
vrs_status seed_buffers(vrs_engine *e, int32_t batch, int64_t M, int64_t cap, cudaStream_t s) {
    TRY(e->smp_ids.ensure((size_t)M * 4));
    TRY(e->smp_count.ensure(8));
    TRY(e->smp_cand.ensure((size_t)batch * cap * 8));
    const size_t before = e->smp_cnt.bytes;
    TRY(e->smp_cnt.ensure((size_t)batch * 4));
    if (e->smp_cnt.bytes != before) CK(cudaMemsetAsync(e->smp_cnt.p, 0, e->smp_cnt.bytes, s));
    return VRS_OK;
}
int seed_grid(const vrs_engine *e, int nqt, int G, int64_t S) {
    // at most the full pass's grid (its global heap buffers are reused)
    return (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)G, e->n_sm / nqt, S / 512}));
}
// Sample pass of the tensor plans.  Without a bound, a CTA's heaps take
// nearly every key of its first tiles, and while the bound is loose the
// lanes of a warp (one query each) keep diverging into heap insertions.
// This pass seeds the per-query bound before the full pass: the selected
// rows among evenly spaced rows (about 1/16 of the selection) go through the
// same kernel with the same arithmetic, so their composites equal the full
// pass's, and each query's bound becomes one past the k'-th smallest of them.
// The k' best selected rows lie at or below it, so the full pass keeps every
// row it needs.  Used where the epilogue bounds the pass: BF16 MASK_GEMM
// with at least kSeedMinRows selected rows per CTA, and E4M3 (k' = 16k
// candidates through global append buffers) on either plan from
// kSeedMinRowsE4M3.  Measured slower, and so not used: BF16 COMPACT_GEMM
// (bound by its row gathers) and the batched launch (bound by its per-query
// range tests).  p: the shared predicate; M: the evenly spaced rows probed;
// S: the selected rows expected among them.
// Enqueues three kernels (the caller counts them).
vrs_status run_seed_pass(vrs_engine *e, const UmmaArgs &full, int dt, int nqt, int G, int64_t M,
                         int64_t S, const PredArg &p, int kp, cudaStream_t s) {
    M = std::max<int64_t>(1, std::min<int64_t>(M, e->n));
    const int Gs = seed_grid(e, nqt, G, S);
    const int64_t cap = (int64_t)Gs * kp;
    TRY(seed_buffers(e, full.B, M, cap, s));
    CK(cudaMemsetAsync(e->smp_count.p, 0, 8, s));
    CK(launch_sample_ids(attr_arg(e), e->n, p, M, e->smp_ids.as<int32_t>(),
                         e->smp_count.as<int64_t>(), s));
    UmmaArgs a = full;
    a.ids = e->smp_ids.as<const int32_t>();
    a.bitmap = nullptr;
    a.count_dev = e->smp_count.as<const int64_t>();
    a.use_tma_x = 0;
    a.out = e->smp_cand.as<uint64_t>();
    a.out_cnt = e->smp_cnt.as<int32_t>();
    a.out_cap = cap;
    CK(launch_umma(a, dt, nqt * Gs, s));
    CK(launch_seed_bound(e->smp_cand.as<const uint64_t>(), cap, e->smp_cnt.as<int32_t>(), full.B,
                         kp, full.kq, full.kp_factor, full.tau_g, s));
    return VRS_OK;
}

// Tensor formulation (Sec. 3.1 N:N) on tcgen05: COMPACT_GEMM over the
// gathered ids, or MASK_GEMM over all rows with the bitmap on the scores.
vrs_status query_tensor(vrs_engine *e, const float *q_dev_pad, uint64_t *tau_g,
                        int32_t *cand_cnt, int32_t batch, int plan, const PredArg &p,
                        int64_t count_est, int kp,
                        const int32_t *k_dev, int32_t k_shared, int32_t k_max,
                        vrs_metric metric, vrs_dtype compute, int64_t *oid, float *odist,
                        cudaStream_t s) {
    const int dt = compute == VRS_BF16 ? 1 : 2;
    const int32_t row_bytes = compute == VRS_BF16 ? e->ld * 2 : e->ld;
    const int32_t Bpad = (batch + 127) / 128 * 128;
    const int nqt = Bpad / 128;
    const int64_t rows = plan == VRS_PLAN_MASK_GEMM ? e->n : count_est;
    int G = e->grid_ctas > 0 ? e->grid_ctas : std::max(1, e->n_sm / nqt);
    G = (int)std::min<int64_t>(G, std::max<int64_t>(1, (rows + 1023) / 1024));
    const int grid = nqt * G;
    int ns;
    bool resa, hs;
    size_t smem;
    if (!umma_config(row_bytes, kp, &ns, &resa, &smem, &hs))
        return fail(VRS_EINVAL, "no tensor-core tiling fits k'=%d, row of %d bytes", kp, row_bytes);
    TRY(e->qenc.ensure((size_t)Bpad * row_bytes));
    TRY(e->qnorm.ensure((size_t)batch * 4));
    TRY(e->qscale.ensure((size_t)batch * 4));
    TRY(e->qres.ensure((size_t)batch * 4));
    const int64_t out_cap = (int64_t)G * kp;
    TRY(e->cand.ensure((size_t)batch * out_cap * 8));
    if (!hs) TRY(e->heap_g.ensure(umma_global_buffer_bytes(grid, kp)));
    const bool fp8 = compute == VRS_FP8E4M3;
    // A lossy encoding rarely certifies a first pass of default width at
    // large d: start from a sample of the selection instead (below).
    const bool sampled = e->cert_sample && e->rerank && !e->fb_seed &&
                         e->cert_Rx[compute] > 0.0f && k_max > 0 && kp < kMaxKpWide;
    const bool seed = !sampled && e->seed_bound && !e->fb_seed &&
                      (plan == VRS_PLAN_MASK_GEMM || fp8) &&
                      count_est / G >= (fp8 ? kSeedMinRowsE4M3 : kSeedMinRows);
    set_first_pass(e, fp8 ? kCertE4M3 : kCertBF16, compute, e->qres.as<const float>());

    StageTimer t(e, s);
    t.begin();
    CK(launch_prep_tensor_queries(q_dev_pad, batch, Bpad, e->d, e->ld, dt,
                                  e->qenc.as<unsigned char>(), row_bytes, e->qnorm.as<float>(),
                                  e->qscale.as<float>(), e->qres.as<float>(), s));
    if (e->fb_seed) {
        // widened certifying pass: keep every row whose first-pass key is
        // within this pass's bound of the k-th exact key found so far
        CK(launch_cert_seed(e->fb_seed, e->qnorm.as<const float>(), cert_args(e), metric, batch,
                            tau_g, cand_cnt, s));
        e->launches += 1;
    }
    t.end(VRS_STAGE_PREPARE);
    UmmaArgs a{};
    a.X = dt == 1 ? e->xb.as<const unsigned char>() : e->x8.as<const unsigned char>();
    a.row_bytes = row_bytes;
    a.xnorm = e->norms.as<const float>();
    a.xscale = dt == 2 ? e->s8.as<const float>() : nullptr;
    a.ids = plan == VRS_PLAN_COMPACT_GEMM ? e->ids.as<const int32_t>() : nullptr;
    a.bitmap = plan == VRS_PLAN_MASK_GEMM ? e->bitmap.as<const uint32_t>() : nullptr;
    a.count_dev = e->count_q.as<const int64_t>();
    a.n_rows = e->n;
    a.Q = e->qenc.as<const unsigned char>();
    a.qnorm = e->qnorm.as<const float>();
    a.qscale = dt == 2 ? e->qscale.as<const float>() : nullptr;
    a.B = batch;
    a.metric = metric;
    a.kp = kp;
    a.tau_g = tau_g;
    a.out_cnt = cand_cnt;
    a.out = e->cand.as<uint64_t>();
    a.out_cap = out_cap;
    a.heap_g = hs ? nullptr : e->heap_g.as<uint64_t>();
    a.err = e->err.as<int32_t>();
    a.use_tma_q = make_tmap_2d(&a.tmQ, a.Q, row_bytes, Bpad, 128) ? 1 : 0;
    a.use_tma_x = (!a.ids && make_tmap_2d(&a.tmX, a.X, row_bytes, e->n, 256)) ? 1 : 0;
    if (!e->tma) a.use_tma_q = a.use_tma_x = 0;
    t.begin();
    if (sampled) {
        // Sample-seeded exact pass.  (1) About 1/16 of the selected rows
        // (among evenly spaced rows) go through the same kernel and an exact
        // re-rank: their k-th exact distance D is at least the whole
        // selection's, so every row of the exact top-k has a first-pass key
        // <= D + E.  (2) One full pass keeps exactly those rows (bound seeded
        // at D + E, k' up to kMaxKpWide); its merge certifies the query when
        // it kept them all.
        const double s_est = std::max(1e-6, (double)count_est / (double)e->n);
        const int64_t S = std::max<int64_t>(kSeedMinRowsE4M3, count_est / 16);
        const int64_t M = std::max<int64_t>(
            1, std::min<int64_t>(e->n, std::min<int64_t>(64 * S, std::max<int64_t>(
                                                                   S, (int64_t)(1.25 * S / s_est)))));
        const int Gs = seed_grid(e, nqt, G, S);
        const int64_t cap_s = (int64_t)Gs * kp;
        const int kpw = kMaxKpWide;
        int ns_w;
        bool resa_w, hs_w;
        size_t smem_w;
        if (!umma_config(row_bytes, kpw, &ns_w, &resa_w, &smem_w, &hs_w))
            return fail(VRS_EINVAL, "no tensor-core tiling fits k'=%d", kpw);
        const int64_t out_cap_w = (int64_t)G * kpw;
        TRY(seed_buffers(e, batch, M, cap_s, s));
        TRY(e->cand.ensure((size_t)batch * out_cap_w * 8));
        TRY(e->heap_g.ensure(std::max(umma_global_buffer_bytes(grid, kpw),
                                      hs ? (size_t)0 : umma_global_buffer_bytes(nqt * Gs, kp))));
        TRY(e->fb_oid.ensure((size_t)batch * k_max * 8));
        TRY(e->fb_odist.ensure((size_t)batch * k_max * 4));
        TRY(e->fb_flag.ensure((size_t)batch * 4));
        TRY(e->fb_dup.ensure((size_t)batch * 4));
        CK(cudaMemsetAsync(e->smp_count.p, 0, 8, s));
        CK(launch_sample_ids(attr_arg(e), e->n, p, M, e->smp_ids.as<int32_t>(),
                             e->smp_count.as<int64_t>(), s));
        UmmaArgs as = a;
        as.ids = e->smp_ids.as<const int32_t>();
        as.bitmap = nullptr;
        as.count_dev = e->smp_count.as<const int64_t>();
        as.use_tma_x = 0;
        as.out = e->smp_cand.as<uint64_t>();
        as.out_cnt = e->smp_cnt.as<int32_t>();
        as.out_cap = cap_s;
        as.heap_g = hs ? nullptr : e->heap_g.as<uint64_t>();
        CK(launch_umma(as, dt, nqt * Gs, s));
        MergeArgs m{};
        m.cand = e->smp_cand.as<const uint64_t>();
        m.m = cap_s;
        m.cand_cnt = e->smp_cnt.as<int32_t>();
        m.kp = kp;
        m.k = k_dev;
        m.k_shared = k_shared;
        m.k_max = k_max;
        m.B = batch;
        m.metric = metric;
        m.rerank = 1;
        m.Xf = e->has[VRS_F32] ? e->x32.as<const float>() : nullptr;
        m.Xb = e->has[VRS_F32] ? nullptr : e->xb.as<const uint16_t>();
        m.ld = e->ld;
        m.d = e->d;
        m.Q = q_dev_pad;
        m.ldq = e->ld;
        m.out_ids = e->fb_oid.as<int64_t>();
        m.out_dist = e->fb_odist.as<float>();
        m.reset_tau = tau_g;
        m.stage_cap = (int32_t)std::min<int64_t>(cap_s, 4096);
        m.cert = cert_args(e);
        m.cert_flag = e->fb_flag.as<int32_t>();
        m.cert_dup = e->fb_dup.as<float>();
        m.dup_only = 1;
        CK(launch_merge_rerank(m, s));
        CK(launch_cert_seed(e->fb_dup.as<const float>(), e->qnorm.as<const float>(), cert_args(e),
                            metric, batch, tau_g, cand_cnt, s));
        a.kp = kpw;
        a.out = e->cand.as<uint64_t>();   // (re)allocated above for the wider list
        a.out_cap = out_cap_w;
        a.heap_g = hs_w ? nullptr : e->heap_g.as<uint64_t>();
        CK(launch_umma(a, dt, grid, s));
        t.end(VRS_STAGE_DISTANCE);
        e->launches += 6;   // prep, sample ids, sample pass, sample merge, seed, full pass
        return run_merge(e, q_dev_pad, e->ld, tau_g, cand_cnt, out_cap_w, batch, kpw, k_dev,
                         k_shared, k_max, metric, oid, odist, s);
    }
    if (seed) {
        // about 1/16 of the selection, found among evenly spaced rows
        const double s_est = std::max(1e-6, (double)count_est / (double)e->n);
        const int64_t S = std::max<int64_t>(fp8 ? kSeedMinRowsE4M3 : kSeedMinRows, count_est / 16);
        const int64_t M = std::min<int64_t>(64 * S, std::max<int64_t>(S, (int64_t)(1.25 * S / s_est)));
        TRY(run_seed_pass(e, a, dt, nqt, G, M, S, p, kp, s));
        e->launches += 3;
    }
    CK(launch_umma(a, dt, grid, s));
    t.end(VRS_STAGE_DISTANCE);
    e->launches += 2;
    return run_merge(e, q_dev_pad, e->ld, tau_g, cand_cnt, out_cap, batch, kp, k_dev, k_shared,
                     k_max, metric, oid, odist, s);
}

// Dense-key GEMV form: a key matrix of at most 256 MB and rows the merge
// kernel holds in registers (ld <= 2048).
bool dense_keys_ok(const vrs_engine *e, int32_t batch) {
    return e->dense_keys && (int64_t)batch * e->n * 4 <= ((int64_t)256 << 20) && e->ld <= 2048;
}

// Row stride of the dense key matrix (a multiple of 4 for vector loads).
int64_t keys_ld(const vrs_engine *e) { return (e->n + 3) & ~(int64_t)3; }

// Row stride of the per-chunk minima (one per 128 positions).
int64_t cmin_ld(const vrs_engine *e) { return (e->n + 127) / 128; }

// List capacity of the dense-key merge: room for the chunk minima of up to
// parts * 3072 positions and for the keys of the candidate chunks, within
// the dynamic shared memory a CTA can have next to the kernel's static
// arrays (a query whose candidates overflow is selected from its whole key
// row).
int keys_merge_cap(const vrs_engine *e, int parts, int kp) {
    int64_t cap = e->select_cap;
    if (cap <= 0) cap = std::max<int64_t>({4096, (int64_t)parts * 24 + 64, 4 * (int64_t)kp});
    const int64_t room = (int64_t)keys_merge_max_smem() - (int64_t)keys_merge_smem(kp, 0, e->ld);
    return (int)std::max<int64_t>(1, std::min<int64_t>(cap, room / 8));
}

// Selection from the dense key matrix + exact re-rank + final top-k.
vrs_status run_keys_merge(vrs_engine *e, const float *q_dev, int32_t ldq, uint64_t *tau_g,
                          int32_t *cand_cnt, int32_t batch, int kp, const int32_t *k_dev,
                          int32_t k_shared, int32_t k_max, vrs_metric metric, int cap,
                          int64_t *oid, float *odist, cudaStream_t s) {
    MergeArgs m{};
    m.cand_cnt = cand_cnt;
    m.kp = kp;
    m.k = k_dev;
    m.k_shared = k_shared;
    m.k_max = k_max;
    m.B = batch;
    m.metric = metric;
    m.rerank = e->rerank;
    m.Xf = e->has[VRS_F32] ? e->x32.as<const float>() : nullptr;
    m.Xb = e->has[VRS_F32] ? nullptr : e->xb.as<const uint16_t>();
    m.ld = e->ld;
    m.d = e->d;
    m.Q = q_dev;
    m.ldq = ldq;
    m.out_ids = oid;
    m.out_dist = odist;
    m.reset_tau = tau_g;
    m.reset_count = e->count_q.as<int64_t>();
    m.keys = e->keys.as<const float>();
    m.keys_ld = keys_ld(e);
    m.key_ids = e->ids.as<const int32_t>();
    // the count as the distance pass copied it (it clears the original)
    m.key_count = e->count_q.as<const int64_t>() + 2;
    m.chunk_min = e->cmin.as<const uint32_t>();
    m.cmin_ld = cmin_ld(e);
    m.done = nullptr;
    m.cert = cert_args(e);
    m.cert_flag = e->cur_cflag;
    m.cert_dup = e->cur_cdup;
    if (e->err_to_host) {
        m.err_src = e->err.as<const int32_t>();
        m.err_dst = e->h_err_dev;
    }
    StageTimer t(e, s);
    t.begin();
    CK(launch_keys_merge(m, cap, s));
    t.end(VRS_STAGE_MERGE);
    e->launches += 1;
    return VRS_OK;
}

// Dense-key distance pass: the staged kernel (rows through shared memory,
// one CTA per SM and query group) when enabled and it fits, otherwise the
// register kernel on G row partitions.
bool use_tensor_gemv(const vrs_engine *e, int32_t batch, int x_bf16) {
    return e->tensor_gemv && !x_bf16 && umma_rows_fits(batch, e->ld);
}
bool use_staged_scan(const vrs_engine *e, int32_t batch, int x_bf16) {
    return e->staged_scan && scan_keys_staged_fits(batch, e->ld, x_bf16);
}
bool use_pair_gemv(const vrs_engine *e, int32_t batch, int x_bf16) {
    return e->tensor_gemv && e->pair_copy && !x_bf16 && e->xp.p && umma_pair_fits(batch, e->d);
}
// 0: register CUDA-core kernel, 1: staged CUDA-core kernel, 2: tensor cores
// over the float32 rows (TF32 split), 3: tensor cores over the bf16 pair copy
int keys_kernel(const vrs_engine *e, int32_t batch, int x_bf16) {
    return use_pair_gemv(e, batch, x_bf16)     ? 3
           : use_tensor_gemv(e, batch, x_bf16) ? 2
           : use_staged_scan(e, batch, x_bf16) ? 1
                                                : 0;
}
int keys_cert_kind(const vrs_engine *e, int32_t batch, int x_bf16) {
    const int kk = keys_kernel(e, batch, x_bf16);
    return kk == 3 ? kCertBF16x3 : kk == 2 ? kCertTF32x3 : kCertFFMA;
}
vrs_status run_keys_scan(vrs_engine *e, const ScanArgs &a, int32_t batch, int G, cudaStream_t s) {
    StageTimer t(e, s);
    t.begin();
    const int kk = keys_kernel(e, batch, a.x_bf16);
    if (kk == 3) {
        const int Gt = e->grid_ctas > 0 ? e->grid_ctas : umma_pair_grid(batch, e->n_sm);
        ScanArgs b = a;
        b.wait_test = e->wait_test ? 1 : 0;
        e->wait_test = false;
        CK(launch_umma_pair(b, e->xp.p, Gt, s));
    } else if (kk == 2) {
        const int Gt = e->grid_ctas > 0 ? e->grid_ctas : umma_rows_grid(batch, e->n_sm);
        CK(launch_umma_rows(a, Gt, s));
    } else if (kk == 1) {
        const int nqg = (batch + scan_simt_query_block(batch) - 1) / scan_simt_query_block(batch);
        const int Gs = e->grid_ctas > 0 ? e->grid_ctas : std::max(1, e->n_sm / nqg);
        CK(launch_scan_keys_staged(a, Gs, s));
    } else {
        CK(launch_scan_simt(a, G, s));
    }
    t.end(VRS_STAGE_DISTANCE);
    return VRS_OK;
}

// Distance pass + merge for one batch that shares one predicate.
// Enqueue the dense-key GEMV pipeline (filter -> ids, key matrix, per-query
// selection + merge).  No allocation: every buffer must already be sized.
vrs_status enqueue_gemv_keys(vrs_engine *e, const float *q, uint64_t *tau_g, int32_t *cand_cnt,
                             int32_t batch, const PredArg &p, const PredArg *pdev, int kp,
                             const int32_t *k_dev, int32_t k_shared, int32_t k_max,
                             vrs_metric metric, vrs_dtype compute, int G, int parts,
                             int64_t *oid, float *odist, cudaStream_t s) {
    {
        StageTimer t(e, s);
        t.begin();
        CK(launch_predicate_ids(attr_arg(e), e->n, p, pdev, e->ids.as<int32_t>(),
                                e->count_q.as<int64_t>(), e->n_sm, s));
        t.end(VRS_STAGE_PREDICATE);
    }
    ScanArgs a{};
    a.X = compute == VRS_BF16 ? e->xb.p : e->x32.p;
    a.x_bf16 = compute == VRS_BF16 ? 1 : 0;
    a.ld = e->ld;
    a.d = e->d;
    a.xnorm = e->norms.as<const float>();
    a.ids = e->ids.as<const int32_t>();
    a.count_dev = e->count_q.as<const int64_t>();
    a.n_rows = e->n;
    a.Q = q;
    a.B = batch;
    a.metric = metric;
    a.kp = kp;
    a.tau_g = tau_g;
    a.out_cnt = cand_cnt;
    a.keys_out = e->keys.as<float>();
    a.keys_ld = keys_ld(e);
    a.chunk_min = e->cmin.as<uint32_t>();
    a.cmin_ld = cmin_ld(e);
    a.err = e->err.as<int32_t>();
    a.count_copy = e->count_q.as<int64_t>() + 2;
    set_first_pass(e, keys_cert_kind(e, batch, a.x_bf16), compute, nullptr);
    TRY(run_keys_scan(e, a, batch, G, s));
    e->launches += 2;   // filter and distance pass (the merge counts itself)
    return run_keys_merge(e, q, e->ld, tau_g, cand_cnt, batch, kp, k_dev, k_shared, k_max, metric,
                          keys_merge_cap(e, parts, kp), oid, odist, s);
}

// Graph form: the sequence is run eagerly the first time a shape is seen,
// captured into a CUDA graph the second time, and replayed afterwards.  The
// predicate lives in a device buffer (copied before each launch), so one
// graph serves every predicate of the same shape.
vrs_status gemv_keys_graph(vrs_engine *e, const float *q, uint64_t *tau_g, int32_t *cand_cnt,
                           int32_t batch, const PredArg &p, int kp, const int32_t *k_dev,
                           int32_t k_shared, int32_t k_max, vrs_metric metric, vrs_dtype compute,
                           int G, int parts, int64_t *oid, float *odist, cudaStream_t s) {
    const int cap = keys_merge_cap(e, parts, kp);
    TRY(e->ids.ensure((size_t)e->n * 4));
    {
        const size_t before = e->count_q.bytes;
        TRY(e->count_q.ensure(64));
        if (e->count_q.bytes != before) CK(cudaMemsetAsync(e->count_q.p, 0, e->count_q.bytes, s));
    }
    TRY(e->keys.ensure((size_t)batch * keys_ld(e) * 4));
    TRY(e->cmin.ensure((size_t)batch * cmin_ld(e) * 4));
    TRY(upload_pred(e, p, s));
    const PredArg *pdev = e->pred_dev.as<const PredArg>();
    // a host-buffer call: upload, downloads and the error word in the sequence
    const float *qh = e->io_q_host;
    int64_t *ih = e->io_ids_host;
    float *dh = e->io_dist_host;
    e->io_q_host = nullptr;
    e->io_out_done = ih != nullptr;
    const size_t qbytes = e->io_q_bytes, on = e->io_out_n;
    // zero copy: the kernels read the page-locked queries and write the
    // results into the caller's page-locked buffers through their device
    // addresses (over the CPU-GPU link), so the sequence holds no copies but
    // the error word's
    const bool zc = e->zero_copy && qh && ih && dh && e->io_q_dev && e->io_ids_dev && e->io_dist_dev;
    if (zc) {
        q = e->io_q_dev;
        oid = e->io_ids_dev;
        odist = e->io_dist_dev;
    }
    auto enqueue_all = [&]() -> vrs_status {
        if (qh && !zc) CK(cudaMemcpyAsync(const_cast<float *>(q), qh, qbytes, cudaMemcpyHostToDevice, s));
        // zero copy: the merge kernel also writes the error word to the host
        e->err_to_host = zc && ih && e->h_err_dev;
        const vrs_status st = enqueue_gemv_keys(e, q, tau_g, cand_cnt, batch, p, pdev, kp, k_dev,
                                                k_shared, k_max, metric, compute, G, parts, oid,
                                                odist, s);
        e->err_to_host = false;
        TRY(st);
        if (ih) {
            if (!zc) {
                CK(cudaMemcpyAsync(ih, oid, on * 8, cudaMemcpyDeviceToHost, s));
                CK(cudaMemcpyAsync(dh, odist, on * 4, cudaMemcpyDeviceToHost, s));
                CK(cudaMemcpyAsync(e->h_err, e->err.p, 4, cudaMemcpyDeviceToHost, s));
            }
        }
        return VRS_OK;
    };
    char kb[400];
    snprintf(kb, sizeof kb, "gemv-b%d-kp%d-km%d-ks%d-m%d-c%d-G%d-P%d-S%d-C%lld-q%p-o%p-%p-t%p-k%p-f%p-%p-p%d-h%p-%p-%p-e%llu",
             batch, kp, k_max, k_shared, (int)metric, (int)compute, G, parts,
             keys_kernel(e, batch, compute == VRS_BF16),
             (long long)cap, (const void *)q,
             (void *)oid, (void *)odist, (void *)tau_g, (const void *)k_dev,
             (void *)e->cur_cflag, (void *)e->cur_cdup, (int)e->profile, (const void *)qh,
             (void *)ih, (void *)dh, (unsigned long long)g_ws_epoch);
    const std::string key = kb;
    for (auto &ge : e->graphs) {
        if (ge.key != key || e->wait_test) continue;
        CK(cudaGraphLaunch(ge.exec, s));
        e->launches += 3;   // filter, distance pass, merge
        e->marks.clear();
        for (const auto &m : ge.marks) e->marks.push_back({m.stage, ge.evs[m.a], ge.evs[m.b]});
        return VRS_OK;
    }
    if (e->pending_key != key || e->wait_test) {   // first sighting (or a test hook): eager
        if (!e->wait_test) e->pending_key = key;
        return enqueue_all();
    }
    const int64_t launches0 = e->launches;
    vrs_engine::GraphEntry ge;
    ge.key = key;
    e->capturing = true;
    e->cap = &ge;
    cudaGraph_t g = nullptr;
    vrs_status st = VRS_OK;
    cudaError_t ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        st = enqueue_all();
        ce = cudaStreamEndCapture(s, &g);
    }
    e->capturing = false;
    e->cap = nullptr;
    if (st == VRS_OK && ce == cudaSuccess) ce = cudaGraphInstantiate(&ge.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (st != VRS_OK || ce != cudaSuccess) {
        for (cudaEvent_t ev : ge.evs) cudaEventDestroy(ev);
        if (st != VRS_OK) return st;
        return fail(VRS_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    }
    if (e->graphs.size() >= 8) {
        auto &old = e->graphs.front();
        cudaGraphExecDestroy(old.exec);
        for (cudaEvent_t ev : old.evs) cudaEventDestroy(ev);
        e->graphs.erase(e->graphs.begin());
    }
    e->graphs.push_back(std::move(ge));
    auto &cur = e->graphs.back();
    CK(cudaGraphLaunch(cur.exec, s));
    e->launches = launches0 + 3;
    e->marks.clear();
    for (const auto &m : cur.marks) e->marks.push_back({m.stage, cur.evs[m.a], cur.evs[m.b]});
    return VRS_OK;
}

// Fused FP32 scan (predicate on the fly, bulk row gather) + merge.
vrs_status query_gemv_fused(vrs_engine *e, const float *q_raw, uint64_t *tau_g,
                            int32_t *cand_cnt, int32_t batch, const PredArg &p, int kp,
                            int64_t count_est, const int32_t *k_dev, int32_t k_shared,
                            int32_t k_max, vrs_metric metric, int64_t *oid, float *odist,
                            cudaStream_t s) {
    const int qb = gemv_fused_query_block(batch);
    const int nqg = (batch + qb - 1) / qb;
    // one CTA per SM and query group; the table is split into G ranges
    int G = e->grid_ctas > 0 ? e->grid_ctas : std::max(1, (e->n_sm + nqg - 1) / nqg);
    G = (int)std::min<int64_t>(G, std::max<int64_t>(1, (e->n + 127) / 128));
    const int64_t out_cap = (int64_t)G * kp;
    TRY(e->cand.ensure((size_t)batch * out_cap * 8));
    TRY(e->count.ensure(64));
    GemvArgs a{};
    a.X = e->x32.as<const float>();
    a.ld = e->ld;
    a.d = e->d;
    a.xnorm = e->norms.as<const float>();
    a.attrs = attr_arg(e);
    a.pred = p;
    a.n = e->n;
    a.Q = q_raw;
    a.ldq = e->d;
    a.B = batch;
    a.metric = metric;
    a.kp = kp;
    a.tau_g = tau_g;
    a.out_cnt = cand_cnt;
    a.out = e->cand.as<uint64_t>();
    a.out_cap = out_cap;
    a.count_out = nullptr;
    if (e->profile) {
        CK(cudaMemsetAsync(e->count.p, 0, 8, s));
        a.count_out = e->count.as<int64_t>();
    }
    a.err = e->err.as<int32_t>();
    (void)count_est;
    set_first_pass(e, kCertFFMA, VRS_F32, nullptr);
    StageTimer t(e, s);
    t.begin();
    CK(launch_gemv_fused(a, G, s));
    t.end(VRS_STAGE_DISTANCE);
    e->launches += 1;
    return run_merge(e, q_raw, e->d, tau_g, cand_cnt, out_cap, batch, kp, k_dev, k_shared, k_max,
                     metric, oid, odist, s);
}

// Whole query for a batch that shares one predicate.  q_raw: [batch x d]
// float32 on the device.
vrs_status query_shared(vrs_engine *e, const float *q_raw, uint64_t *tau_g,
                        int32_t *cand_cnt, int32_t batch, const PredArg &p,
                        const int32_t *k_dev, int32_t k_shared, int32_t k_max, vrs_metric metric,
                        vrs_dtype compute, int64_t *oid, float *odist, cudaStream_t s) {
    // Plan and grid from the sampled selectivity; the kernels read the exact
    // count on the device, so no host round trip is needed here.
    const double s_est = estimate_selectivity(e, p);
    const int64_t count = std::min<int64_t>(e->n, (int64_t)std::ceil(s_est * e->n) + 256);
    e->last_count = -1;

    int plan = e->plan_forced >= 0
                   ? e->plan_forced
                   : (e->planner ? planner_choice(e, batch, s_est, k_max, compute)
                                 : fixed_rule(e, batch, s_est, compute));
    if (plan == VRS_PLAN_GEMV && compute == VRS_FP8E4M3)
        return fail(VRS_EINVAL, "the GEMV plan reads float32 or bf16 rows, not FP8");
    if (plan != VRS_PLAN_GEMV && compute == VRS_F32)
        return fail(VRS_EINVAL, "tensor plans compute in BF16 or FP8");
    e->last_plan = plan;

    // E4M3's worst-case error band is too wide to certify a pass of any
    // affordable width (its 3-bit mantissa); with a BF16 copy resident the
    // sample-seeded exact form runs in BF16, which certifies in one pass
    if (compute == VRS_FP8E4M3 && plan != VRS_PLAN_GEMV && e->cert_sample && e->rerank &&
        e->has[VRS_BF16] && !e->fb_seed)
        compute = VRS_BF16;
    const int kp = e->fb_kp > 0 ? e->fb_kp : default_kprime(e, k_max, compute);
    const bool graph_form = plan == VRS_PLAN_GEMV && e->use_graph && s != nullptr &&
                            e->ld == e->d && dense_keys_ok(e, batch) &&
                            !(e->fused_gemv && compute == VRS_F32);
    if (e->io_q_host && !graph_form) {   // only the captured form takes the upload itself
        CK(cudaMemcpyAsync(const_cast<float *>(q_raw), e->io_q_host, e->io_q_bytes,
                           cudaMemcpyHostToDevice, s));
        e->io_q_host = nullptr;
    }
    // A float32 batch too large for the dense key matrix runs in sub-batches
    // that fit it, so it stays on the tensor-core GEMV kernels (each
    // sub-batch re-reads the selected rows; the alternative is the CUDA-core
    // scan with selection inside it)
    if (plan == VRS_PLAN_GEMV && compute == VRS_F32 && e->fb_kp == 0 && !dense_keys_ok(e, batch) &&
        !(e->fused_gemv && compute == VRS_F32) && e->tensor_gemv) {
        int32_t c = 64;
        while (c >= 8 && !(dense_keys_ok(e, c) && keys_kernel(e, c, 0) >= 2)) c >>= 1;
        if (c >= 8 && c < batch) {
            int32_t *cf = e->cur_cflag;
            float *cd = e->cur_cdup;
            int64_t *ioi = e->io_ids_host;
            float *iod = e->io_dist_host;
            e->io_ids_host = nullptr;   // the results go down once, after every sub-batch
            e->io_dist_host = nullptr;
            vrs_status st = VRS_OK;
            for (int32_t off = 0; off < batch && st == VRS_OK; off += c) {
                const int32_t nb = std::min(c, batch - off);
                e->cur_cflag = cf + off;
                e->cur_cdup = cd + off;
                st = query_shared(e, q_raw + (int64_t)off * e->d, tau_g + off, cand_cnt + off, nb, p,
                                  k_dev ? k_dev + off : nullptr, k_shared, k_max, metric, compute,
                                  oid + (int64_t)off * k_max, odist + (int64_t)off * k_max, s);
            }
            e->cur_cflag = cf;
            e->cur_cdup = cd;
            e->io_ids_host = ioi;
            e->io_dist_host = iod;
            e->last_plan = VRS_PLAN_GEMV;
            return st;
        }
    }
    if (plan == VRS_PLAN_GEMV && e->fused_gemv && compute == VRS_F32 &&
        gemv_fused_smem(gemv_fused_query_block(batch), e->ld, kp) <= 227 * 1024)
        return query_gemv_fused(e, q_raw, tau_g, cand_cnt, batch, p, kp, count, k_dev, k_shared,
                                k_max, metric, oid, odist, s);

    // queries padded to the row stride (rows already at the stride are used
    // as they are; the search state was left cleared by the previous merge)
    const float *q_dev_pad = q_raw;
    if (e->ld != e->d) {
        TRY(e->qpad.ensure((size_t)batch * e->ld * 4));
        StageTimer tp(e, s);
        tp.begin();
        CK(launch_prep_queries(q_raw, batch, e->d, e->qpad.as<float>(), e->ld, tau_g, cand_cnt, s));
        tp.end(VRS_STAGE_PREPARE);
        e->launches += 1;
        q_dev_pad = e->qpad.as<const float>();
    }
    const int qb = scan_simt_query_block(batch);
    const int nqg0 = (batch + qb - 1) / qb;
    if (plan == VRS_PLAN_GEMV && e->use_graph && s != nullptr && q_dev_pad == q_raw &&
        dense_keys_ok(e, batch)) {
        // captured-graph form of the dense-key GEMV pipeline
        // persistent: the CTAs one wave holds (3 per SM for small query
        // groups, 2 at 8-16 queries), split over the query groups
        const int per_sm = qb >= 8 ? 2 : 3;
        int G = e->grid_ctas > 0 ? e->grid_ctas
                                 : std::max(1, (per_sm * e->n_sm + nqg0 - 1) / nqg0);
        G = (int)std::min<int64_t>(G, std::max<int64_t>(1, (count + 127) / 128));
        const int parts = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (count + 3071) / 3072));
        return gemv_keys_graph(e, q_raw, tau_g, cand_cnt, batch, p, kp, k_dev, k_shared, k_max,
                               metric, compute, G, parts, oid, odist, s);
    }
    if (plan == VRS_PLAN_MASK_GEMM) TRY(run_filter(e, p, s));
    else TRY(run_filter_ids(e, p, s));
    if (plan != VRS_PLAN_GEMV)
        return query_tensor(e, q_dev_pad, tau_g, cand_cnt, batch, plan, p, count, kp, k_dev,
                            k_shared, k_max, metric, compute, oid, odist, s);

    const int nqg = (batch + qb - 1) / qb;
    // Dense-key form for small batches: the distance pass writes every key
    // into a [batch x rows] matrix (L2-resident) and the merge selects the
    // k' best of each row; no selection inside the scan.
    const bool keys_mode = dense_keys_ok(e, batch);
    int G = e->grid_ctas > 0 ? e->grid_ctas : std::max(1, (8 * e->n_sm + nqg - 1) / nqg);
    G = (int)std::min<int64_t>(G, std::max<int64_t>(1, (count + (keys_mode ? 127 : 255)) /
                                                           (keys_mode ? 128 : 256)));
    const int parts = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (count + 3071) / 3072));
    const int64_t out_cap = keys_mode ? 0 : (int64_t)G * kp;
    if (keys_mode) {
        TRY(e->keys.ensure((size_t)batch * keys_ld(e) * 4));
        TRY(e->cmin.ensure((size_t)batch * cmin_ld(e) * 4));
    } else {
        TRY(e->cand.ensure((size_t)batch * out_cap * 8));
    }

    ScanArgs a{};
    a.X = compute == VRS_BF16 ? e->xb.p : e->x32.p;
    a.x_bf16 = compute == VRS_BF16 ? 1 : 0;
    a.ld = e->ld;
    a.d = e->d;
    a.xnorm = e->norms.as<const float>();
    a.ids = e->ids.as<const int32_t>();
    a.bitmap = nullptr;
    a.count_dev = e->count_q.as<const int64_t>();
    a.n_rows = e->n;
    a.Q = q_dev_pad;
    a.B = batch;
    a.metric = metric;
    a.kp = kp;
    a.tau_g = tau_g;
    a.out_cnt = cand_cnt;
    a.out = e->cand.as<uint64_t>();
    a.out_cap = out_cap;
    a.keys_out = keys_mode ? e->keys.as<float>() : nullptr;
    a.keys_ld = keys_ld(e);
    a.chunk_min = keys_mode ? e->cmin.as<uint32_t>() : nullptr;
    a.cmin_ld = cmin_ld(e);
    a.err = e->err.as<int32_t>();
    if (keys_mode) a.count_copy = e->count_q.as<int64_t>() + 2;
    set_first_pass(e, keys_mode ? keys_cert_kind(e, batch, a.x_bf16) : kCertFFMA, compute,
                   nullptr);
    if (keys_mode) {
        TRY(run_keys_scan(e, a, batch, G, s));
    } else {
        StageTimer t(e, s);
        t.begin();
        CK(launch_scan_simt(a, G, s));
        t.end(VRS_STAGE_DISTANCE);
    }
    e->launches += 1;
    if (keys_mode)
        return run_keys_merge(e, q_dev_pad, e->ld, tau_g, cand_cnt, batch, kp, k_dev, k_shared,
                              k_max, metric, keys_merge_cap(e, parts, kp), oid, odist, s);
    return run_merge(e, q_dev_pad, e->ld, tau_g, cand_cnt, out_cap, batch, kp, k_dev, k_shared,
                     k_max, metric, oid, odist, s);
}

// ---------------------------------------------------------------------------
// Batched launch for per-query predicates (one launch of the tensor kernel
// over every query of the batch; each query's own conjunction is applied to
// its scores in the epilogue).
// ---------------------------------------------------------------------------

// Pack per-query conjunctions into inclusive ranges over a shared column set.
// Returns false if more than kMaxQCols distinct columns are used.
bool pack_query_ranges(const std::vector<PredArg> &pa, std::vector<int32_t> &cols,
                       std::vector<int32_t> &rng) {
    cols.clear();
    for (const auto &p : pa)
        for (int t = 0; t < p.n_terms; ++t)
            if (std::find(cols.begin(), cols.end(), p.col[t]) == cols.end()) cols.push_back(p.col[t]);
    if ((int)cols.size() > kMaxQCols) return false;
    const int nc = (int)cols.size();
    rng.assign(pa.size() * nc * 2, 0);
    for (size_t b = 0; b < pa.size(); ++b) {
        for (int c = 0; c < nc; ++c) {
            int64_t lo = INT32_MIN, hi = INT32_MAX;   // inclusive
            for (int t = 0; t < pa[b].n_terms; ++t) {
                if (pa[b].col[t] != cols[c]) continue;
                lo = std::max<int64_t>(lo, pa[b].lo[t]);
                hi = std::min<int64_t>(hi, (int64_t)pa[b].hi[t] - 1);
            }
            if (lo > hi) { lo = 1; hi = 0; }   // empty
            rng[(b * nc + c) * 2] = (int32_t)lo;
            rng[(b * nc + c) * 2 + 1] = (int32_t)hi;
        }
    }
    return true;
}

// Enqueue the batched kernel sequence (prep, tensor prep, tensor scan, merge).
vrs_status enqueue_batched(vrs_engine *e, const float *qsrc, int32_t batch, int nqc,
                           const int32_t *cols, const int32_t *kd, int32_t k_max, int kp,
                           vrs_metric metric, vrs_dtype compute, int G, int64_t *oid,
                           float *odist, cudaStream_t s) {
    const int dt = compute == VRS_BF16 ? 1 : 2;
    const int32_t row_bytes = compute == VRS_BF16 ? e->ld * 2 : e->ld;
    const int32_t Bpad = (batch + 127) / 128 * 128;
    const int nqt = Bpad / 128;
    const int grid = nqt * G;
    int ns;
    bool resa, hs;
    size_t smem;
    if (!umma_config(row_bytes, kp, &ns, &resa, &smem, &hs))
        return fail(VRS_EINVAL, "no tensor-core tiling fits k'=%d", kp);
    const int64_t out_cap = (int64_t)G * kp;
    uint64_t *tau_g = e->tau_g.as<uint64_t>();
    int32_t *cand_cnt = e->cand_cnt.as<int32_t>();
    CK(launch_prep_queries(qsrc, batch, e->d, e->qpad.as<float>(), e->ld, tau_g, cand_cnt, s));
    CK(launch_prep_tensor_queries(e->qpad.as<const float>(), batch, Bpad, e->d, e->ld, dt,
                                  e->qenc.as<unsigned char>(), row_bytes, e->qnorm.as<float>(),
                                  e->qscale.as<float>(), e->qres.as<float>(), s));
    set_first_pass(e, dt == 2 ? kCertE4M3 : kCertBF16, compute, e->qres.as<const float>());
    UmmaArgs a{};
    a.X = dt == 1 ? e->xb.as<const unsigned char>() : e->x8.as<const unsigned char>();
    a.row_bytes = row_bytes;
    a.xnorm = e->norms.as<const float>();
    a.xscale = dt == 2 ? e->s8.as<const float>() : nullptr;
    a.ids = nullptr;
    a.bitmap = nullptr;
    a.count_dev = nullptr;
    a.n_rows = e->n;
    a.Q = e->qenc.as<const unsigned char>();
    a.qnorm = e->qnorm.as<const float>();
    a.qscale = dt == 2 ? e->qscale.as<const float>() : nullptr;
    a.B = batch;
    a.metric = metric;
    a.kp = kp;
    a.tau_g = tau_g;
    a.out_cnt = cand_cnt;
    a.out = e->cand.as<uint64_t>();
    a.out_cap = out_cap;
    a.heap_g = hs ? nullptr : e->heap_g.as<uint64_t>();
    a.err = e->err.as<int32_t>();
    a.nqc = nqc;
    for (int c = 0; c < nqc; ++c) a.qcol[c] = e->attr[cols[c]].as<const int32_t>();
    a.qrange = e->qrange.as<const int32_t>();
    // each query keeps and re-ranks the width its own k needs
    a.kq = kd;
    a.kp_factor = kprime_factor(e, compute);
    a.use_tma_q = make_tmap_2d(&a.tmQ, a.Q, row_bytes, Bpad, 128) ? 1 : 0;
    a.use_tma_x = make_tmap_2d(&a.tmX, a.X, row_bytes, e->n, 256) ? 1 : 0;
    if (!e->tma) a.use_tma_q = a.use_tma_x = 0;
    CK(launch_umma(a, dt, grid, s));
    MergeArgs m{};
    m.cand = e->cand.as<const uint64_t>();
    m.m = out_cap;
    m.cand_cnt = cand_cnt;
    m.kp = kp;
    m.k = kd;
    m.k_shared = k_max;
    m.k_max = k_max;
    m.B = batch;
    m.metric = metric;
    m.rerank = e->rerank;
    m.Xf = e->has[VRS_F32] ? e->x32.as<const float>() : nullptr;
    m.Xb = e->has[VRS_F32] ? nullptr : e->xb.as<const uint16_t>();
    m.ld = e->ld;
    m.d = e->d;
    m.Q = e->qpad.as<const float>();
    m.ldq = e->ld;
    m.out_ids = oid;
    m.out_dist = odist;
    m.stage_cap = (int32_t)std::min<int64_t>(out_cap, 4096);
    m.kp_factor = kprime_factor(e, compute);
    // every merge leaves the per-query state cleared for the next query
    m.reset_tau = tau_g;
    m.reset_count = e->count_q.p ? e->count_q.as<int64_t>() : nullptr;
    m.cert = cert_args(e);
    m.cert_flag = e->cflag.as<int32_t>();
    m.cert_dup = e->cdup.as<float>();
    CK(launch_merge_rerank(m, s));
    return VRS_OK;
}

// A page-locked slot of at least `bytes` for this call's uploads (waits
// for the copies last issued from it); pin_done records their completion.
vrs_status pin_take(vrs_engine *e, size_t bytes, unsigned char **out) {
    auto &ps = e->pin[e->pin_next];
    if (ps.used) CK(cudaEventSynchronize(ps.ev));
    if (ps.bytes < bytes) {
        if (ps.p) cudaFreeHost(ps.p);
        ps.p = nullptr;
        ps.bytes = 0;
        const size_t want = std::max<size_t>(bytes, (size_t)1 << 20);
        if (fault_alloc() || cudaHostAlloc(&ps.p, want, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            ps.p = nullptr;
            return fail(VRS_ENOMEM, "page-locked staging of %zu bytes failed", want);
        }
        ps.bytes = want;
    }
    if (!ps.ev) CK(cudaEventCreateWithFlags(&ps.ev, cudaEventDisableTiming));
    *out = static_cast<unsigned char *>(ps.p);
    return VRS_OK;
}
vrs_status pin_done(vrs_engine *e, cudaStream_t s) {
    auto &ps = e->pin[e->pin_next];
    CK(cudaEventRecord(ps.ev, s));
    ps.used = true;
    e->pin_next ^= 1;
    return VRS_OK;
}

// ---------------------------------------------------------------------------
// Cell plan (k_cells.cu): a batch whose predicates are conjunctions of ranges
// on the two columns of the grid vrs_build_grid made (or have no terms).
// The host plans from the predicates and the grid's cell sizes alone: each
// query's rectangle of cells and its fully covered bins, its key row (the
// chunks of its cells, from the summed-area table), the cells' query counts
// (a 2-D difference array) and the work items.  The device fills the
// (query, cell) pairs, runs the GEMM over the items and the dense-key merge
// over the per-query rows.  Sub-batches keep the key matrix under
// kCellKeyBytes.
// ---------------------------------------------------------------------------
constexpr int64_t kCellKeyBytes = (int64_t)48 << 30;

bool cells_eligible(const vrs_engine *e, const std::vector<PredArg> &pa, vrs_dtype compute) {
    if (!e->cell_plan || !e->grid.valid || compute != VRS_BF16 || !e->has[VRS_BF16] || !e->rerank)
        return false;
    for (const auto &p : pa)
        for (int t = 0; t < p.n_terms; ++t)
            if (p.col[t] != e->grid.col[0] && p.col[t] != e->grid.col[1]) return false;
    return true;
}

// A query's inclusive ranges on the grid's two columns, its cells and the
// fully covered bins (rect: b0lo b0hi b1lo b1hi f0lo f0hi f1lo f1hi; an
// empty range gives an empty rectangle).
void cell_rect(const vrs_engine *e, const PredArg &p, int32_t *rect, int32_t *rng) {
    const auto &G = e->grid;
    int64_t lo[2] = {INT32_MIN, INT32_MIN}, hi[2] = {INT32_MAX, INT32_MAX};
    for (int t = 0; t < p.n_terms; ++t) {
        const int c = p.col[t] == G.col[0] ? 0 : 1;
        lo[c] = std::max<int64_t>(lo[c], p.lo[t]);
        hi[c] = std::min<int64_t>(hi[c], (int64_t)p.hi[t] - 1);
    }
    const bool empty = lo[0] > hi[0] || lo[1] > hi[1];
    for (int c = 0; c < 2; ++c) {
        const auto &E = G.edge[c];
        const int nb = G.nb[c];
        auto bin = [&](int64_t v) {
            return std::max(0, std::min(nb - 1, (int)(std::upper_bound(E.begin(), E.end(), v) - E.begin()) - 1));
        };
        int blo = bin(lo[c]), bhi = bin(hi[c]);
        int flo = E[blo] >= lo[c] ? blo : blo + 1;
        int fhi = E[bhi + 1] - 1 <= hi[c] ? bhi : bhi - 1;
        if (empty) blo = 0, bhi = -1, flo = 0, fhi = -1;
        rect[2 * c] = blo;
        rect[2 * c + 1] = bhi;
        rect[4 + 2 * c] = flo;
        rect[4 + 2 * c + 1] = fhi;
        rng[2 * c] = (int32_t)std::max<int64_t>(lo[c], INT32_MIN);
        rng[2 * c + 1] = (int32_t)std::min<int64_t>(hi[c], INT32_MAX);
    }
}

int64_t rect_chunks(const vrs_engine *e, const int32_t *r) {
    if (r[1] < r[0] || r[3] < r[2]) return 0;
    const int w = e->grid.nb[1] + 1;
    const auto &S = e->grid.sat;
    return S[(size_t)(r[1] + 1) * w + r[3] + 1] - S[(size_t)r[0] * w + r[3] + 1] -
           S[(size_t)(r[1] + 1) * w + r[2]] + S[(size_t)r[0] * w + r[2]];
}

// One sub-batch: queries qa .. qb of the batch.
// width: queries per work item (64 or 128); stages: the GEMM's row stages (0: most)
vrs_status enqueue_cells(vrs_engine *e, const float *qsrc, int32_t qa, int32_t qb,
                         const std::vector<int32_t> &rect, const std::vector<int32_t> &rng,
                         const int32_t *k_dev, int32_t k_shared, int32_t k_max, int kp,
                         vrs_metric metric, int width, int stages, int64_t *oid, float *odist,
                         cudaStream_t s) {
    const auto &G = e->grid;
    const int32_t nb = qb - qa;
    const int nb0 = G.nb[0], nb1 = G.nb[1], ncell = nb0 * nb1;
    const int32_t row_bytes = e->ld * 2;
    const int32_t Bpad = (nb + 127) / 128 * 128;
    // key rows, pairs per cell, items
    std::vector<int64_t> qc0((size_t)nb + 1, 0);
    std::vector<int64_t> diff((size_t)(nb0 + 1) * (nb1 + 1), 0);
    for (int32_t i = 0; i < nb; ++i) {
        const int32_t *r = &rect[(size_t)(qa + i) * 8];
        qc0[(size_t)i + 1] = qc0[(size_t)i] + rect_chunks(e, r);
        if (r[1] < r[0] || r[3] < r[2]) continue;
        diff[(size_t)r[0] * (nb1 + 1) + r[2]] += 1;
        diff[(size_t)r[0] * (nb1 + 1) + r[3] + 1] -= 1;
        diff[(size_t)(r[1] + 1) * (nb1 + 1) + r[2]] -= 1;
        diff[(size_t)(r[1] + 1) * (nb1 + 1) + r[3] + 1] += 1;
    }
    const int64_t chunks = qc0[(size_t)nb];
    std::vector<int32_t> entry0((size_t)ncell + 1, 0);
    std::vector<CellItem> items;
    for (int b0 = 0; b0 < nb0; ++b0)
        for (int b1 = 0; b1 < nb1; ++b1) {
            int64_t v = diff[(size_t)b0 * (nb1 + 1) + b1];
            if (b0 > 0) v += diff[(size_t)(b0 - 1) * (nb1 + 1) + b1];
            if (b1 > 0) v += diff[(size_t)b0 * (nb1 + 1) + b1 - 1];
            if (b0 > 0 && b1 > 0) v -= diff[(size_t)(b0 - 1) * (nb1 + 1) + b1 - 1];
            diff[(size_t)b0 * (nb1 + 1) + b1] = v;   // prefix sums in place: v = pairs of cell
            const int c = b0 * nb1 + b1;
            const int32_t cnt = G.nch[(size_t)c] > 0 ? (int32_t)v : 0;
            entry0[(size_t)c + 1] = entry0[(size_t)c] + cnt;
            for (int32_t j = 0; j < cnt; j += width)
                items.push_back(CellItem{c, entry0[(size_t)c] + j, std::min(width, cnt - j), 0});
        }
    // the work queue takes the largest items first (row tiles x padded queries)
    std::stable_sort(items.begin(), items.end(), [&](const CellItem &x, const CellItem &y) {
        const int64_t cx = (int64_t)G.nch[(size_t)x.cell] * (x.nq + 16);
        const int64_t cy = (int64_t)G.nch[(size_t)y.cell] * (y.nq + 16);
        return cx > cy;
    });
    const int64_t pairs = entry0[(size_t)ncell];
    // stage events: the uploads, query preparation and pair lists; the GEMM
    // alone; the merge (the host work above sits outside every stage)
    StageTimer t(e, s);
    t.begin();
    // buffers
    TRY(e->c_rect.ensure((size_t)nb * 32));
    TRY(e->c_qrange.ensure((size_t)nb * 16));
    TRY(e->c_qchunk0.ensure(((size_t)nb + 1) * 8));
    TRY(e->c_entry0.ensure(((size_t)ncell + 1) * 4));
    TRY(e->c_cursor.ensure((size_t)ncell * 8 + 16));
    TRY(e->c_entries.ensure(std::max<size_t>(1, (size_t)pairs) * sizeof(CellEntry)));
    TRY(e->c_items.ensure(std::max<size_t>(1, items.size()) * sizeof(CellItem)));
    TRY(e->c_keys.ensure(std::max<size_t>(1, (size_t)chunks) * 128 * 4));
    TRY(e->c_cmin.ensure(std::max<size_t>(1, (size_t)chunks) * 4));
    TRY(e->c_crow.ensure(std::max<size_t>(1, (size_t)chunks) * 4));
    TRY(e->qpad.ensure((size_t)nb * e->ld * 4));
    TRY(e->qenc.ensure((size_t)Bpad * row_bytes));
    TRY(e->qnorm.ensure((size_t)nb * 4));
    TRY(e->qscale.ensure((size_t)nb * 4));
    TRY(e->qres.ensure((size_t)nb * 4));
    {
        // one page-locked staging area, one copy per array
        const size_t sz[5] = {(size_t)nb * 32, (size_t)nb * 16, qc0.size() * 8, entry0.size() * 4,
                              items.size() * sizeof(CellItem)};
        const void *src[5] = {&rect[(size_t)qa * 8], &rng[(size_t)qa * 4], qc0.data(), entry0.data(),
                              items.data()};
        void *dst[5] = {e->c_rect.p, e->c_qrange.p, e->c_qchunk0.p, e->c_entry0.p, e->c_items.p};
        size_t tot = 0;
        for (size_t x : sz) tot += (x + 15) & ~(size_t)15;
        unsigned char *h;
        TRY(pin_take(e, tot, &h));
        for (int i = 0; i < 5; ++i) {
            if (sz[i] == 0) continue;
            memcpy(h, src[i], sz[i]);
            CK(cudaMemcpyAsync(dst[i], h, sz[i], cudaMemcpyHostToDevice, s));
            h += (sz[i] + 15) & ~(size_t)15;
        }
        TRY(pin_done(e, s));
    }
    CK(cudaMemsetAsync(e->c_cursor.p, 0, (size_t)ncell * 8 + 16, s));   // (+ the queue counter)

    uint64_t *tau_g = e->tau_g.as<uint64_t>() + qa;
    int32_t *cand_cnt = e->cand_cnt.as<int32_t>() + qa;
    CK(launch_prep_queries(qsrc + (int64_t)qa * e->d, nb, e->d, e->qpad.as<float>(), e->ld, tau_g,
                           cand_cnt, s));
    CK(launch_prep_tensor_queries(e->qpad.as<const float>(), nb, Bpad, e->d, e->ld, 1,
                                  e->qenc.as<unsigned char>(), row_bytes, e->qnorm.as<float>(),
                                  e->qscale.as<float>(), e->qres.as<float>(), s));
    set_first_pass(e, kCertBF16, VRS_BF16, e->qres.as<const float>());
    if (pairs > 0)
        CK(launch_cell_fill(e->c_rect.as<const int32_t>(), nb, e->c_qchunk0.as<const int64_t>(),
                            G.nch_d.as<const int32_t>(), nb1, ncell, e->c_entry0.as<const int32_t>(),
                            e->c_cursor.as<int32_t>(), e->c_entries.as<CellEntry>(), s));
    t.end(VRS_STAGE_PREPARE);
    if (!items.empty()) {
        CellArgs a{};
        a.tmX = G.tmX;
        a.Q = e->qenc.as<const unsigned char>();
        a.row_bytes = G.row_bytes;
        a.q_bytes = row_bytes;
        a.metric = metric;
        a.qnorm = e->qnorm.as<const float>();
        a.xnorm = G.ng.as<const float>();
        a.a0 = G.g0.as<const int32_t>();
        a.a1 = G.g1.as<const int32_t>();
        a.qrange = e->c_qrange.as<const int32_t>();
        a.cell_off = G.off_d.as<const int64_t>();
        a.items = e->c_items.as<const CellItem>();
        a.n_items = (int32_t)items.size();
        a.entries = e->c_entries.as<const CellEntry>();
        a.keys = e->c_keys.as<float>();
        a.chunk_min = e->c_cmin.as<uint32_t>();
        a.chunk_row = e->c_crow.as<int32_t>();
        a.item_next = e->c_cursor.as<int32_t>() + 2 * ncell;
        a.err = e->err.as<int32_t>();
        const int grid = (int)std::min<int64_t>(e->n_sm, (int64_t)items.size());
        t.begin();
        CK(launch_cells_gemm(a, e->grid_ctas > 0 ? e->grid_ctas : grid, stages, s));
        t.end(VRS_STAGE_DISTANCE);
        e->launches += 1;
    }
    MergeArgs m{};
    m.kp = kp;
    m.k = k_dev ? k_dev + qa : nullptr;
    m.k_shared = k_shared;
    m.k_max = k_max;
    m.B = nb;
    m.metric = metric;
    m.rerank = e->rerank;
    m.Xf = e->has[VRS_F32] ? e->x32.as<const float>() : nullptr;
    m.Xb = e->has[VRS_F32] ? nullptr : e->xb.as<const uint16_t>();
    m.ld = e->ld;
    m.d = e->d;
    m.Q = e->qpad.as<const float>();
    m.ldq = e->ld;
    m.out_ids = oid + (int64_t)qa * k_max;
    m.out_dist = odist + (int64_t)qa * k_max;
    m.reset_tau = tau_g;
    m.keys = e->c_keys.as<const float>();
    m.chunk_min = e->c_cmin.as<const uint32_t>();
    m.row_chunk0 = e->c_qchunk0.as<const int64_t>();
    m.chunk_row = e->c_crow.as<const int32_t>();
    m.row_ids = G.ids.as<const int32_t>();
    m.cert = cert_args(e);
    m.cert_flag = e->cur_cflag + qa;
    m.cert_dup = e->cur_cdup + qa;
    t.begin();
    CK(launch_keys_merge(m, keys_merge_cap(e, 0, kp), s));
    t.end(VRS_STAGE_MERGE);
    e->launches += 4;   // prep, tensor prep, fill, merge
    return VRS_OK;
}

vrs_status query_cells(vrs_engine *e, const float *qsrc, int32_t batch,
                       const std::vector<PredArg> &pa, const int32_t *k, int32_t n_k, int32_t k_max,
                       vrs_metric metric, int64_t *oid, float *odist, cudaStream_t s) {
    std::vector<int32_t> rect((size_t)batch * 8), rng((size_t)batch * 4);
    for (int32_t i = 0; i < batch; ++i)
        cell_rect(e, pa[pa.size() == 1 ? 0 : (size_t)i], &rect[(size_t)i * 8], &rng[(size_t)i * 4]);
    // per-query k on the device
    const int32_t *k_dev = nullptr;
    if (n_k == batch) {
        TRY(e->kdev.ensure((size_t)batch * 4));
        unsigned char *h;
        TRY(pin_take(e, (size_t)batch * 4, &h));
        memcpy(h, k, (size_t)batch * 4);
        CK(cudaMemcpyAsync(e->kdev.p, h, (size_t)batch * 4, cudaMemcpyHostToDevice, s));
        TRY(pin_done(e, s));
        k_dev = e->kdev.as<const int32_t>();
    }
    // candidate width: the bf16 products are exact and only the float32
    // accumulation (and, for a float32 table, the rounding of the rows)
    // separates first-pass keys from exact ones
    const int kp = e->bf16_is_master ? std::min(kMaxKp, std::max(k_max + 8, 16))
                                     : default_kprime(e, k_max, VRS_BF16);
    auto run = [&](int width, int stages) -> vrs_status {
        int32_t qa = 0;
        int64_t acc = 0;
        for (int32_t i = 0; i <= batch; ++i) {
            const int64_t c = i < batch ? rect_chunks(e, &rect[(size_t)i * 8]) : 0;
            if (i == batch || (i > qa && (acc + c) * 512 > kCellKeyBytes)) {
                TRY(enqueue_cells(e, qsrc, qa, i, rect, rng, k_dev, n_k == 1 ? k[0] : k_max, k_max,
                                  kp, metric, width, stages, oid, odist, s));
                qa = i;
                acc = 0;
            }
            acc += c;
        }
        return VRS_OK;
    };
    // tile autotuning: the first batch of a shape runs every (queries per
    // item, row stages) pair once and keeps the fastest (each run computes
    // the same exact result); later batches of the shape use it
    char keybuf[160];
    snprintf(keybuf, sizeof keybuf, "cells-b%d-n%lld-d%d-g%dx%d-m%d-k%d", batch, (long long)e->n,
             e->d, e->grid.nb[0], e->grid.nb[1], (int)metric, k_max);
    const std::string key = keybuf;
    int choice = -1;
    for (auto &kv : e->tuned)
        if (kv.first == key) choice = kv.second;
    static const int kWidth[2] = {128, 64}, kStages[3] = {8, 6, 4};
    if (choice < 0 && !e->profile) {
        cudaEvent_t a0, a1;
        CK(cudaEventCreate(&a0));
        CK(cudaEventCreate(&a1));
        float best = 1e30f;
        for (int c = 0; c < 6; ++c) {
            CK(cudaEventRecord(a0, s));
            TRY(run(kWidth[c / 3], kStages[c % 3]));
            CK(cudaEventRecord(a1, s));
            CK(cudaEventSynchronize(a1));
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, a0, a1));
            if (ms < best) {
                best = ms;
                choice = c;
            }
        }
        cudaEventDestroy(a0);
        cudaEventDestroy(a1);
        e->tuned.push_back({key, choice});
    }
    if (choice < 0) choice = 0;
    TRY(run(kWidth[choice / 3], kStages[choice % 3]));
    e->last_plan = VRS_PLAN_CELLS;
    return VRS_OK;
}

vrs_status query_batched(vrs_engine *e, const float *qsrc, int32_t batch,
                         const std::vector<PredArg> &pa, const int32_t *k, int32_t n_k,
                         int32_t k_max, vrs_metric metric, vrs_dtype compute, int64_t *oid,
                         float *odist, cudaStream_t s, bool *done) {
    *done = false;
    std::vector<int32_t> cols;
    if (!pack_query_ranges(pa, cols, e->h_qrange)) return VRS_OK;   // caller falls back
    const int nqc = (int)cols.size();
    const int kp = default_kprime(e, k_max, compute);
    const int32_t row_bytes = compute == VRS_BF16 ? e->ld * 2 : e->ld;
    const int32_t Bpad = (batch + 127) / 128 * 128;
    const int nqt = Bpad / 128;
    int ns;
    bool resa, hs;
    size_t smem;
    if (!umma_config(row_bytes, kp, &ns, &resa, &smem, &hs)) return VRS_OK;

    // device-side inputs of the sequence (fixed buffers, so a captured graph
    // stays valid while the shape is unchanged)
    TRY(e->qrange.ensure(std::max<size_t>(e->h_qrange.size() * 4, 16)));
    if (!e->h_qrange.empty())
        CK(cudaMemcpyAsync(e->qrange.p, e->h_qrange.data(), e->h_qrange.size() * 4,
                           cudaMemcpyHostToDevice, s));
    TRY(e->kdev.ensure((size_t)batch * 4));
    std::vector<int32_t> kh(batch);
    for (int i = 0; i < batch; ++i) kh[i] = n_k == 1 ? k[0] : k[i];
    CK(cudaMemcpyAsync(e->kdev.p, kh.data(), (size_t)batch * 4, cudaMemcpyHostToDevice, s));
    TRY(e->qpad.ensure((size_t)batch * e->ld * 4));
    TRY(e->qenc.ensure((size_t)Bpad * row_bytes));
    TRY(e->qnorm.ensure((size_t)batch * 4));
    TRY(e->qscale.ensure((size_t)batch * 4));
    TRY(e->qres.ensure((size_t)batch * 4));

    // grid: autotuned per shape among {1, 2, 4} waves of one CTA per SM
    char keybuf[160];
    snprintf(keybuf, sizeof keybuf, "b%d-n%lld-d%d-dt%d-kp%d-nc%d-m%d", batch, (long long)e->n,
             e->d, (int)compute, kp, nqc, (int)metric);
    const std::string key = keybuf;
    int G = 0;
    for (auto &kv : e->tuned)
        if (kv.first == key) G = kv.second;
    const int G1 = std::max(1, e->n_sm / nqt);
    const int Gmax_rows = (int)std::max<int64_t>(1, (e->n + 1023) / 1024);
    const int cand_G[3] = {std::min(G1, Gmax_rows), std::min(2 * G1, Gmax_rows),
                           std::min(4 * G1, Gmax_rows)};
    // the largest grid this call may launch (a forced grid included)
    const int Gbig = std::max({cand_G[0], cand_G[1], cand_G[2], e->grid_ctas});
    TRY(e->cand.ensure((size_t)batch * Gbig * kp * 8));
    if (!hs) TRY(e->heap_g.ensure(umma_global_buffer_bytes(nqt * Gbig, kp)));
    if (e->grid_ctas > 0) G = e->grid_ctas;
    if (G == 0) {
        cudaEvent_t a0, a1;
        CK(cudaEventCreate(&a0));
        CK(cudaEventCreate(&a1));
        float best = 1e30f;
        for (int ci = 0; ci < 3; ++ci) {
            if (ci > 0 && cand_G[ci] == cand_G[ci - 1]) continue;
            CK(cudaEventRecord(a0, s));
            TRY(enqueue_batched(e, qsrc, batch, nqc, cols.data(), e->kdev.as<const int32_t>(), k_max,
                                kp, metric, compute, cand_G[ci], oid, odist, s));
            CK(cudaEventRecord(a1, s));
            CK(cudaEventSynchronize(a1));
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, a0, a1));
            if (ms < best) {
                best = ms;
                G = cand_G[ci];
            }
        }
        cudaEventDestroy(a0);
        cudaEventDestroy(a1);
        e->tuned.push_back({key, G});
    }
    e->last_plan = VRS_PLAN_MASK_GEMM;

    StageTimer t(e, s);
    t.begin();
    if (e->use_graph && !e->profile) {
        char gk[256];
        snprintf(gk, sizeof gk, "%s-G%d-q%p-o%p-%p-e%llu", key.c_str(), G, (const void *)qsrc,
                 (void *)oid, (void *)odist, (unsigned long long)g_ws_epoch);
        if (!e->graph || e->graph_key != gk) {
            if (e->graph) {
                cudaGraphExecDestroy(e->graph);
                e->graph = nullptr;
            }
            cudaStream_t cs;
            CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t g;
            CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            vrs_status st = enqueue_batched(e, qsrc, batch, nqc, cols.data(),
                                            e->kdev.as<const int32_t>(), k_max, kp, metric, compute,
                                            G, oid, odist, cs);
            cudaError_t ce = cudaStreamEndCapture(cs, &g);
            cudaStreamDestroy(cs);
            if (st != VRS_OK) return st;
            if (ce != cudaSuccess) return fail(VRS_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&e->graph, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) {
                e->graph = nullptr;
                return fail(VRS_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(ce));
            }
            e->graph_key = gk;
        }
        CK(cudaGraphLaunch(e->graph, s));
        e->launches += 4;   // the graph holds the four kernels
    } else {
        TRY(enqueue_batched(e, qsrc, batch, nqc, cols.data(), e->kdev.as<const int32_t>(), k_max,
                            kp, metric, compute, G, oid, odist, s));
        e->launches += 4;
    }
    t.end(VRS_STAGE_DISTANCE);
    *done = true;
    return VRS_OK;
}

// ---------------------------------------------------------------------------
// Certification fallback.  A merge that re-ranks appended candidates (the
// tensor plans, the in-scan GEMV selection) flags every query it could not
// certify (CertArgs).  Those queries are run again, as a sub-batch, until
// certified:
//   1. a wider tensor pass (BF16 when that copy is resident, else the same
//      encoding) whose per-query bound starts at T = D + E, so it keeps every
//      row that can still belong to the top-k, with k' up to kMaxKpWide;
//   2. the dense-key GEMV plan over the float32 (or bf16 master) rows, whose
//      merge widens itself until certified.
// ---------------------------------------------------------------------------

// Run the queries idx[0..m) of the current batch (rows of q_raw [* x d], k
// from k_dev or k_shared) as one sub-batch under plan/dtype; results go to
// their rows of oid/odist when certified.  Returns the still-uncertified
// queries in *left (indices into the batch).
vrs_status run_subset(vrs_engine *e, const float *q_raw, const std::vector<int32_t> &idx,
                      const PredArg &p, const int32_t *k_dev, int32_t k_shared, int32_t k_max,
                      vrs_metric metric, vrs_dtype dtype, int plan, int kp_wide, bool seed,
                      int64_t *oid, float *odist, cudaStream_t s, std::vector<int32_t> *left) {
    const int32_t m = (int32_t)idx.size();
    left->clear();
    if (m == 0) return VRS_OK;
    TRY(e->fb_idx.ensure((size_t)m * 4));
    TRY(e->fb_q.ensure((size_t)m * e->d * 4));
    TRY(e->fb_dup.ensure((size_t)m * 4));
    TRY(e->fb_k.ensure((size_t)m * 4));
    TRY(e->fb_oid.ensure((size_t)m * k_max * 8));
    TRY(e->fb_odist.ensure((size_t)m * k_max * 4));
    TRY(e->fb_flag.ensure((size_t)m * 4));
    TRY(e->fb_dup2.ensure((size_t)m * 4));
    CK(cudaMemcpyAsync(e->fb_idx.p, idx.data(), (size_t)m * 4, cudaMemcpyHostToDevice, s));
    const int32_t *di = e->fb_idx.as<const int32_t>();
    CK(launch_gather_rows_f32(q_raw, e->d, di, m, e->fb_q.as<float>(), s));
    if (seed)
        CK(launch_gather_rows_f32(e->cdup.as<const float>(), 1, di, m, e->fb_dup.as<float>(), s));
    if (k_dev)
        CK(launch_gather_rows_f32(reinterpret_cast<const float *>(k_dev), 1, di, m,
                                  e->fb_k.as<float>(), s));
    // the sub-batch's own flags; the plan, width and seed of this pass
    int32_t *cf = e->cur_cflag;
    float *cd = e->cur_cdup;
    const int pf = e->plan_forced, lp = e->last_plan;
    const bool ug = e->use_graph, dk = e->dense_keys, fg = e->fused_gemv;
    if (plan == VRS_PLAN_GEMV) {   // the form whose merge certifies itself
        e->dense_keys = true;
        e->fused_gemv = false;
    }
    e->cur_cflag = e->fb_flag.as<int32_t>();
    e->cur_cdup = e->fb_dup2.as<float>();
    e->plan_forced = plan;
    e->use_graph = false;
    e->fb_kp = kp_wide;
    e->fb_seed = seed ? e->fb_dup.as<const float>() : nullptr;
    e->rerank_merge = false;
    const vrs_status st =
        query_shared(e, e->fb_q.as<const float>(), e->tau_g.as<uint64_t>(),
                     e->cand_cnt.as<int32_t>(), m, p,
                     k_dev ? reinterpret_cast<const int32_t *>(e->fb_k.p) : nullptr, k_shared, k_max,
                     metric, dtype, e->fb_oid.as<int64_t>(), e->fb_odist.as<float>(), s);
    e->cur_cflag = cf;
    e->cur_cdup = cd;
    e->plan_forced = pf;
    e->last_plan = lp;   // the plan reported is the first pass's
    e->use_graph = ug;
    e->dense_keys = dk;
    e->fused_gemv = fg;
    e->fb_kp = 0;
    e->fb_seed = nullptr;
    TRY(st);
    CK(launch_scatter_topk(e->fb_oid.as<const int64_t>(), e->fb_odist.as<const float>(), di,
                           e->fb_flag.as<const int32_t>(), m, k_max, oid, odist, s));
    std::vector<int32_t> fl((size_t)m);
    CK(cudaMemcpyAsync(fl.data(), e->fb_flag.p, (size_t)m * 4, cudaMemcpyDeviceToHost, s));
    TRY(check_device_error(e, s));   // synchronises the stream
    for (int32_t i = 0; i < m; ++i)
        if (fl[(size_t)i] == 1) left->push_back(idx[(size_t)i]);
    return VRS_OK;
}

// Count the flags of the last self-certified pass (waits for it).
vrs_status flush_cert(vrs_engine *e) {
    if (e->cert_lazy_n <= 0) return VRS_OK;
    std::vector<int32_t> fl((size_t)e->cert_lazy_n);
    CK(cudaStreamSynchronize(e->cert_lazy_s));
    CK(cudaMemcpy(fl.data(), e->cert_lazy, fl.size() * 4, cudaMemcpyDeviceToHost));
    for (int32_t f : fl) e->cert_count[f == 2 ? 1 : 0] += 1;
    e->cert_lazy_n = 0;
    return VRS_OK;
}

// Queries per sub-batch of the dense-key GEMV fallback (its key matrix must
// fit the dense-key limit).
int32_t gemv_chunk(const vrs_engine *e) {
    const int64_t per = (int64_t)((e->n + 3) & ~(int64_t)3) * 4;
    return (int32_t)std::max<int64_t>(1, std::min<int64_t>(64, ((int64_t)256 << 20) / per));
}

// After a pass over `batch` queries (flags in cur_cflag): certify or re-run
// every flagged query.  p: the shared predicate, or NULL with per_query (one
// predicate per query, each re-run alone).
vrs_status certify_batch(vrs_engine *e, const float *q_raw, int32_t batch, const PredArg *p,
                         const std::vector<PredArg> *per_query, const int32_t *k_dev,
                         int32_t k_shared, int32_t k_max, vrs_metric metric, vrs_dtype compute,
                         int64_t *oid, float *odist, cudaStream_t s) {
    if (!e->rerank) return VRS_OK;
    if (!e->rerank_merge) {   // every merge certified itself: count later
        e->cert_lazy = e->cur_cflag;
        e->cert_lazy_n = batch;
        e->cert_lazy_s = s;
        return VRS_OK;
    }
    std::vector<int32_t> fl((size_t)batch);
    CK(cudaMemcpyAsync(fl.data(), e->cur_cflag, (size_t)batch * 4, cudaMemcpyDeviceToHost, s));
    TRY(check_device_error(e, s));   // synchronises the stream
    std::vector<int32_t> U;
    for (int32_t b = 0; b < batch; ++b) {
        if (fl[(size_t)b] == 1) U.push_back(b);
        else e->cert_count[fl[(size_t)b] == 2 ? 1 : 0] += 1;
    }
    if (U.empty()) return VRS_OK;
    // the cdup values the seeded pass starts from are those of this batch
    if (e->cur_cdup != e->cdup.as<float>()) {
        TRY(e->cdup.ensure((size_t)batch * 4));
        CK(cudaMemcpyAsync(e->cdup.p, e->cur_cdup, (size_t)batch * 4, cudaMemcpyDeviceToDevice, s));
    }
    const vrs_dtype exact = e->has[VRS_F32] ? VRS_F32 : VRS_BF16;
    std::vector<int32_t> left;
    if (p && compute != VRS_F32) {
        // 1. wider tensor pass, seeded by the certificate's bound
        const vrs_dtype wd = e->has[VRS_BF16] ? VRS_BF16 : compute;
        const double s_est = estimate_selectivity(e, *p);
        const int plan = fixed_rule(e, (int32_t)U.size(), s_est, wd);
        TRY(run_subset(e, q_raw, U, *p, k_dev, k_shared, k_max, metric, wd, plan, kMaxKpWide,
                       true, oid, odist, s, &left));
        e->cert_count[2] += (int64_t)(U.size() - left.size());
        U.swap(left);
    }
    // 2. exact dense-key GEMV (certifies itself by widening in the merge)
    const int32_t chunk = p ? gemv_chunk(e) : 1;
    for (size_t off = 0; off < U.size(); off += (size_t)chunk) {
        std::vector<int32_t> part(U.begin() + off, U.begin() + std::min(U.size(), off + chunk));
        const PredArg &pp = p ? *p : (*per_query)[(size_t)part[0]];
        TRY(run_subset(e, q_raw, part, pp, k_dev, k_shared, k_max, metric, exact, VRS_PLAN_GEMV, 0,
                       false, oid, odist, s, &left));
        if (!left.empty())
            return fail(VRS_EINTERNAL, "query %d could not be certified exact (the dense-key "
                                       "form does not fit: n=%lld, ld=%d)",
                        left[0], (long long)e->n, e->ld);
        e->cert_count[3] += (int64_t)part.size();
    }
    return VRS_OK;
}

// query_shared followed by the certification of its queries.
vrs_status query_shared_exact(vrs_engine *e, const float *q_raw, int32_t batch, const PredArg &p,
                              const int32_t *k_dev, int32_t k_shared, int32_t k_max,
                              vrs_metric metric, vrs_dtype compute, int64_t *oid, float *odist,
                              cudaStream_t s) {
    TRY(flush_cert(e));   // this pass reuses the flag buffer
    TRY(e->cflag.ensure((size_t)batch * 4));
    TRY(e->cdup.ensure((size_t)batch * 4));
    e->cur_cflag = e->cflag.as<int32_t>();
    e->cur_cdup = e->cdup.as<float>();
    e->rerank_merge = false;
    TRY(query_shared(e, q_raw, e->tau_g.as<uint64_t>(), e->cand_cnt.as<int32_t>(), batch, p, k_dev,
                     k_shared, k_max, metric, compute, oid, odist, s));
    return certify_batch(e, q_raw, batch, &p, nullptr, k_dev, k_shared, k_max, metric, compute, oid,
                         odist, s);
}

}  // namespace

namespace vrs {
// Records the thread-local message vrs_last_error() returns (for entry
// points defined in other translation units).
vrs_status set_error(vrs_status st, const char *msg) { return fail(st, "%s", msg); }
}  // namespace vrs

extern "C" {

const char *vrs_version(void) { return "0.1.0"; }

const char *vrs_last_error(void) { return g_err.c_str(); }

vrs_status vrs_create(int device, vrs_engine **out) {
    if (!out) return fail(VRS_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return fail(VRS_ECUDA, "cudaGetDeviceCount failed: %s", cudaGetErrorString(ce));
    }
    if (device < 0 || device >= ndev)
        return fail(VRS_EINVAL, "device %d out of range (%d devices)", device, ndev);
    DeviceGuard g(device);
    vrs_engine *e = new (std::nothrow) vrs_engine();
    if (!e) return fail(VRS_ENOMEM, "host allocation failed");
    e->device = device;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) e->n_sm = prop.multiProcessorCount;
    if (cudaMallocHost(&e->h_count, 64) != cudaSuccess ||
        cudaMallocHost(&e->h_err, 64) != cudaSuccess) {
        if (e->h_count) cudaFreeHost(e->h_count);
        delete e;
        return fail(VRS_ENOMEM, "cudaMallocHost failed");
    }
    if (e->err.ensure(64) != VRS_OK || cudaMemset(e->err.p, 0, 64) != cudaSuccess) {
        cudaFreeHost(e->h_count);
        cudaFreeHost(e->h_err);
        delete e;
        return fail(VRS_ENOMEM, "device allocation failed");
    }
    if (cudaHostGetDevicePointer(reinterpret_cast<void **>(&e->h_err_dev), e->h_err, 0) !=
        cudaSuccess) {
        cudaGetLastError();
        e->h_err_dev = nullptr;   // the error word then comes down by a copy
    }
    // the learned plan model shipped with the library (VRS_PLANNER: another
    // file, or "none"); any failure keeps the fixed rule
    {
        std::string path;
        const char *env = std::getenv("VRS_PLANNER");
        if (env) {
            path = env;
        } else {
            Dl_info info{};
            if (dladdr(reinterpret_cast<void *>(&vrs_create), &info) && info.dli_fname) {
                path = info.dli_fname;
                const size_t slash = path.rfind('/');
                path = (slash == std::string::npos ? std::string(".") : path.substr(0, slash)) +
                       "/data/planner_gb300.bin";
            }
        }
        if (!path.empty() && path != "none") {
            const std::string keep = g_err;   // a missing file is not this call's error
            if (vrs_planner_load(e, path.c_str()) != VRS_OK) g_err = keep;
        }
    }
    *out = e;
    return VRS_OK;
}

vrs_status vrs_destroy(vrs_engine *e) {
    if (!e) return VRS_OK;
    DeviceGuard g(e->device);
    cudaDeviceSynchronize();
    DevBuf *bufs[] = {&e->x32, &e->xp, &e->xb, &e->x8, &e->s8, &e->norms, &e->bitmap, &e->tile_counts,
                      &e->tile_offsets, &e->count, &e->ids, &e->qin, &e->qpad, &e->cand,
                      &e->oid, &e->odist, &e->staging, &e->tau_g, &e->cand_cnt, &e->count_q, &e->qenc,
                      &e->qnorm, &e->qscale, &e->heap_g, &e->err, &e->keys, &e->cmin,
                      &e->pred_dev, &e->qrange, &e->kdev,
                      &e->smp_ids, &e->smp_count, &e->smp_cand, &e->smp_cnt,
                      &e->xn_max, &e->rcount, &e->roff, &e->rids, &e->rdist,
                      &e->jq, &e->jqa, &e->jbm, &e->jtc, &e->jto, &e->jcnt, &e->jqids,
                      &e->jgq, &e->joid, &e->jodist, &e->uids, &e->udist,
                      &e->stats, &e->cflag, &e->cdup, &e->qres, &e->fb_idx, &e->fb_q,
                      &e->fb_dup, &e->fb_k, &e->fb_oid, &e->fb_odist, &e->fb_flag, &e->fb_dup2};
    for (DevBuf *b : bufs) b->release();
    for (auto &a : e->attr) a.release();
    e->grid.release();
    for (auto &ps : e->pin) {
        if (ps.p) cudaFreeHost(ps.p);
        if (ps.ev) cudaEventDestroy(ps.ev);
    }
    for (DevBuf *b : {&e->c_rect, &e->c_qchunk0, &e->c_entry0, &e->c_cursor, &e->c_entries,
                      &e->c_items, &e->c_qrange, &e->c_keys, &e->c_cmin, &e->c_crow})
        b->release();
    for (cudaEvent_t ev : e->ev_pool) cudaEventDestroy(ev);
    if (e->own) cudaStreamDestroy(e->own);
    for (auto &ge : e->graphs) {
        if (ge.exec) cudaGraphExecDestroy(ge.exec);
        for (cudaEvent_t ev : ge.evs) cudaEventDestroy(ev);
    }
    e->pred_dev.release();
    for (cudaEvent_t ev : e->pred_ev)
        if (ev) cudaEventDestroy(ev);
    if (e->pred_pin) cudaFreeHost(e->pred_pin);
    if (e->h_rcount) cudaFreeHost(e->h_rcount);
    if (e->graph) cudaGraphExecDestroy(e->graph);
    e->qrange.release();
    e->kdev.release();
    if (e->h_count) cudaFreeHost(e->h_count);
    if (e->h_err) cudaFreeHost(e->h_err);
    delete e;
    return VRS_OK;
}

vrs_status vrs_load_vectors(vrs_engine *e, const void *x, int64_t n, int32_t d,
                            vrs_dtype in_dtype, uint32_t copies, int x_on_device,
                            void *stream) {
    NvtxRange nvtx_range("vrs_load_vectors");
    if (!e || !x) return fail(VRS_EINVAL, "engine or x is NULL");
    if (n < 1 || n > 0x7fffffffLL) return fail(VRS_EINVAL, "n=%lld out of range", (long long)n);
    if (d < 1 || d > 4096) return fail(VRS_EINVAL, "d=%d out of range (1..4096)", d);
    if (in_dtype != VRS_F32 && in_dtype != VRS_BF16)
        return fail(VRS_EINVAL, "input dtype must be F32 or BF16");
    if (copies & ~7u) return fail(VRS_EINVAL, "copies mask 0x%x has unknown bits", copies);
    if (in_dtype == VRS_BF16) copies |= 1u << VRS_BF16;
    if (in_dtype == VRS_F32) copies |= 1u << VRS_F32;
    DeviceGuard g(e->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t ld = round_up(d, 16);
    e->n = 0;
    e->grid.release();
    for (auto &f : e->attr_loaded) f = false;
    e->sel_valid = false;
    e->xn_max_valid = false;
    for (auto &h : e->has) h = false;

    // source on device (staging copy if it came from the host)
    const void *src = x;
    const size_t esz = in_dtype == VRS_F32 ? 4 : 2;
    if (!x_on_device) {
        TRY(e->staging.ensure((size_t)n * d * esz));
        CK(cudaMemcpyAsync(e->staging.p, x, (size_t)n * d * esz, cudaMemcpyHostToDevice, s));
        src = e->staging.p;
    }
    if (copies & (1u << VRS_F32)) {
        TRY(e->x32.ensure((size_t)n * ld * 4));
        if (in_dtype == VRS_F32)
            CK(launch_copy_f32((const float *)src, n, d, e->x32.as<float>(), ld, s));
        else
            CK(launch_bf16_to_f32((const uint16_t *)src, n, d, e->x32.as<float>(), ld, s));
        e->has[VRS_F32] = true;
    } else {
        e->x32.release();
    }
    if (e->has[VRS_F32] && e->pair_copy && e->tensor_gemv) {
        const int32_t ldp = pair_ld(d);
        TRY(e->xp.ensure((size_t)n * ldp * 4));
        CK(launch_f32_to_pair(e->x32.as<const float>(), n, d, ld, e->xp.as<uint16_t>(), ldp, s));
    } else {
        e->xp.release();
    }
    if (copies & (1u << VRS_BF16)) {
        TRY(e->xb.ensure((size_t)n * ld * 2));
        if (in_dtype == VRS_BF16)
            CK(launch_copy_bf16((const uint16_t *)src, n, d, e->xb.as<uint16_t>(), ld, s));
        else
            CK(launch_f32_to_bf16((const float *)src, n, d, d, e->xb.as<uint16_t>(), ld, s));
        e->has[VRS_BF16] = true;
    } else {
        e->xb.release();
    }
    if (copies & (1u << VRS_FP8E4M3)) {
        if (!e->has[VRS_F32])
            return fail(VRS_EINVAL, "the FP8 copy is encoded from the float32 copy; set its bit");
        TRY(e->x8.ensure((size_t)n * ld));
        TRY(e->s8.ensure((size_t)n * 4));
        CK(launch_f32_to_e4m3(e->x32.as<const float>(), n, d, ld, e->x8.as<uint8_t>(), ld,
                              e->s8.as<float>(), s));
        e->has[VRS_FP8E4M3] = true;
    } else {
        e->x8.release();
        e->s8.release();
    }
    TRY(e->norms.ensure((size_t)n * 4));
    if (in_dtype == VRS_F32)
        CK(launch_norms_f32(e->x32.as<const float>(), n, d, ld, e->norms.as<float>(), s));
    else
        CK(launch_norms_bf16(e->xb.as<const uint16_t>(), n, d, ld, e->norms.as<float>(), s));
    e->bf16_is_master = in_dtype == VRS_BF16;
    // certificate statistics: A = max ||x|| of the re-rank copy (the float32
    // copy, else the bf16 master) and each encoding's max residual
    TRY(e->stats.ensure(64));
    CK(cudaMemsetAsync(e->stats.p, 0, 64, s));
    float st[6] = {0, 0, 0, 0, 0, 0};
    if (e->has[VRS_F32]) {
        const int dt_b = (e->has[VRS_BF16] && !e->bf16_is_master) ? 1 : 0;
        CK(launch_encoding_stats(e->x32.as<const float>(), n, d, ld, dt_b,
                                 e->xb.as<const uint16_t>(), nullptr, nullptr,
                                 e->stats.as<float>(), s));
        if (e->has[VRS_FP8E4M3])
            CK(launch_encoding_stats(e->x32.as<const float>(), n, d, ld, 2, nullptr,
                                     e->x8.as<const uint8_t>(), e->s8.as<const float>(),
                                     e->stats.as<float>() + 2, s));
    } else {
        CK(launch_max_f32(e->norms.as<const float>(), n, e->stats.as<float>() + 4, s));
    }
    CK(cudaMemcpyAsync(st, e->stats.p, sizeof st, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    e->cert_A = e->has[VRS_F32] ? st[0] : sqrtf(st[4]) * 1.0000005f;
    e->cert_Rx[VRS_F32] = 0.0f;
    e->cert_Rx[VRS_BF16] = (e->has[VRS_F32] && !e->bf16_is_master) ? st[1] : 0.0f;
    e->cert_Rx[VRS_FP8E4M3] = st[3];
    e->staging.release();
    e->n = n;
    e->d = d;
    e->ld = ld;
    return VRS_OK;
}

int32_t vrs_float_key(float v) {
    if (std::isnan(v)) return INT32_MAX;
    uint32_t u;
    std::memcpy(&u, &v, 4);
    const int32_t mag = (int32_t)(u & 0x7fffffffu);   // |v| orders like its bits
    return (u >> 31) ? -mag : mag;
}

vrs_status vrs_load_attribute_f32(vrs_engine *e, int32_t col, const float *a, int64_t n,
                                  int a_on_device, void *stream) {
    if (!e || !a) return fail(VRS_EINVAL, "engine or attribute pointer is NULL");
    if (n < 1 || n > 0x7fffffffLL) return fail(VRS_EINVAL, "n=%lld out of range", (long long)n);
    std::vector<float> host;
    const float *src = a;
    if (a_on_device) {
        DeviceGuard g(e->device);
        host.resize((size_t)n);
        CK(cudaMemcpy(host.data(), a, (size_t)n * 4, cudaMemcpyDeviceToHost));
        src = host.data();
    }
    std::vector<int32_t> keys((size_t)n);
    for (int64_t i = 0; i < n; ++i) keys[(size_t)i] = vrs_float_key(src[i]);
    return vrs_load_attribute(e, col, keys.data(), n, 0, stream);
}

vrs_status vrs_load_attribute(vrs_engine *e, int32_t col, const int32_t *a, int64_t n,
                              int a_on_device, void *stream) {
    if (!e || !a) return fail(VRS_EINVAL, "engine or attribute pointer is NULL");
    if (col < 0 || col >= kMaxCols) return fail(VRS_EINVAL, "column %d out of range", col);
    if (e->n == 0) return fail(VRS_ESTATE, "load the vectors first");
    if (n != e->n) return fail(VRS_EINVAL, "attribute length %lld != %lld rows", (long long)n, (long long)e->n);
    DeviceGuard g(e->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (e->grid.valid && (e->grid.col[0] == col || e->grid.col[1] == col)) e->grid.release();
    TRY(e->attr[col].ensure((size_t)n * 4 + 16));
    CK(cudaMemcpyAsync(e->attr[col].p, a, (size_t)n * 4,
                       a_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    const int64_t S = std::min<int64_t>(n, kSampleRows);
    auto &smp = e->attr_sample[col];
    smp.resize((size_t)S);
    for (int64_t j = 0; j < S; ++j) {
        const int64_t i = j * n / S;
        if (a_on_device)
            CK(cudaMemcpy(&smp[(size_t)j], e->attr[col].as<int32_t>() + i, 4, cudaMemcpyDeviceToHost));
        else
            smp[(size_t)j] = a[i];
    }
    e->attr_loaded[col] = true;
    e->sel_valid = false;
    return VRS_OK;
}

vrs_status vrs_build_grid(vrs_engine *e, int32_t col0, int32_t col1, int32_t bins, void *stream) {
    NvtxRange nvtx_range("vrs_build_grid");
    if (!e) return fail(VRS_EINVAL, "engine is NULL");
    if (e->n == 0) return fail(VRS_ESTATE, "no vectors loaded");
    if (col0 < 0 || col0 >= kMaxCols || col1 < 0 || col1 >= kMaxCols || col0 == col1)
        return fail(VRS_EINVAL, "columns %d and %d must be two distinct columns", col0, col1);
    if (!e->attr_loaded[col0] || !e->attr_loaded[col1])
        return fail(VRS_ESTATE, "columns %d and %d must be loaded", col0, col1);
    if (!e->has[VRS_BF16]) return fail(VRS_ESTATE, "the grid needs the bf16 copy");
    const int32_t gld = std::max<int32_t>(e->ld, 64);   // clustered rows: at least one 128-byte K block
    if (!cells_fit(gld * 2)) return fail(VRS_EINVAL, "d=%d is too large for the cell plan", e->d);
    if (bins < 0 || bins > kGridMaxBins) return fail(VRS_EINVAL, "bins=%d out of 0..%d", bins, kGridMaxBins);
    DeviceGuard g(e->device);
    cudaStream_t s = (cudaStream_t)stream;
    auto &G = e->grid;
    G.release();
    const int64_t n = e->n;
    // about 2048 rows per cell by default
    const int want = bins > 0 ? bins
                              : std::max(1, std::min(kGridMaxBins, (int)std::sqrt((double)n / 2048.0)));
    const int cols[2] = {col0, col1};
    DevBuf ed[2], cell, counts, cursor;
    struct Temps {   // freed on every return
        DevBuf *b[5];
        ~Temps() {
            for (DevBuf *x : b) x->release();
        }
    } temps{{&ed[0], &ed[1], &cell, &counts, &cursor}};
    for (int c = 0; c < 2; ++c) {
        // bin boundaries at quantiles of the column's host sample (repeated
        // values give fewer bins)
        std::vector<int32_t> smp = e->attr_sample[cols[c]];
        std::sort(smp.begin(), smp.end());
        auto &E = G.edge[c];
        E.assign(1, (int64_t)INT32_MIN);
        for (int b = 1; b < want && !smp.empty(); ++b) {
            const int64_t v = smp[(size_t)b * smp.size() / (size_t)want];
            if (v > E.back()) E.push_back(v);
        }
        E.push_back((int64_t)INT32_MAX + 1);
        G.nb[c] = (int)E.size() - 1;
        G.col[c] = cols[c];
        std::vector<int32_t> inner(E.begin() + 1, E.end() - 1);
        TRY(ed[c].ensure(std::max<size_t>(4, inner.size() * 4)));
        if (!inner.empty())
            CK(cudaMemcpyAsync(ed[c].p, inner.data(), inner.size() * 4, cudaMemcpyHostToDevice, s));
    }
    const int ncell = G.nb[0] * G.nb[1];
    TRY(cell.ensure((size_t)n * 4));
    TRY(counts.ensure((size_t)ncell * 4));
    TRY(cursor.ensure((size_t)ncell * 4));
    CK(cudaMemsetAsync(counts.p, 0, (size_t)ncell * 4, s));
    CK(cudaMemsetAsync(cursor.p, 0, (size_t)ncell * 4, s));
    CK(launch_grid_cells(e->attr[col0].as<const int32_t>(), e->attr[col1].as<const int32_t>(), n,
                         ed[0].as<const int32_t>(), G.nb[0], ed[1].as<const int32_t>(), G.nb[1],
                         cell.as<int32_t>(), counts.as<int32_t>(), s));
    std::vector<int32_t> cnt((size_t)ncell);
    CK(cudaMemcpyAsync(cnt.data(), counts.p, (size_t)ncell * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    G.off.assign((size_t)ncell + 1, 0);
    G.nch.assign((size_t)ncell, 0);
    for (int c = 0; c < ncell; ++c) {
        G.off[(size_t)c + 1] = G.off[(size_t)c] + cnt[(size_t)c];
        G.nch[(size_t)c] = (cnt[(size_t)c] + 127) / 128;
    }
    const int w = G.nb[1] + 1;
    G.sat.assign((size_t)(G.nb[0] + 1) * w, 0);
    for (int b0 = 0; b0 < G.nb[0]; ++b0)
        for (int b1 = 0; b1 < G.nb[1]; ++b1)
            G.sat[(size_t)(b0 + 1) * w + b1 + 1] = G.nch[(size_t)b0 * G.nb[1] + b1] +
                                                  G.sat[(size_t)b0 * w + b1 + 1] +
                                                  G.sat[(size_t)(b0 + 1) * w + b1] -
                                                  G.sat[(size_t)b0 * w + b1];
    TRY(G.off_d.ensure(G.off.size() * 8));
    TRY(G.nch_d.ensure(G.nch.size() * 4));
    CK(cudaMemcpyAsync(G.off_d.p, G.off.data(), G.off.size() * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(G.nch_d.p, G.nch.data(), G.nch.size() * 4, cudaMemcpyHostToDevice, s));
    TRY(G.ids.ensure((size_t)n * 4));
    CK(launch_grid_scatter(cell.as<const int32_t>(), n, G.off_d.as<const int64_t>(),
                           cursor.as<int32_t>(), G.ids.as<int32_t>(), s));
    TRY(G.xg.ensure((size_t)n * gld * 2));
    TRY(G.ng.ensure((size_t)n * 4));
    TRY(G.g0.ensure((size_t)n * 4));
    TRY(G.g1.ensure((size_t)n * 4));
    CK(launch_grid_gather(G.ids.as<const int32_t>(), n, e->xb.as<const uint16_t>(), e->ld, gld,
                          e->norms.as<const float>(), e->attr[col0].as<const int32_t>(),
                          e->attr[col1].as<const int32_t>(), G.xg.as<uint16_t>(), G.ng.as<float>(),
                          G.g0.as<int32_t>(), G.g1.as<int32_t>(), s));
    G.row_bytes = gld * 2;
    if (!make_tmap_2d(&G.tmX, G.xg.p, (uint64_t)gld * 2, (uint64_t)n, 128))
        return fail(VRS_ECUDA, "tensor map of the clustered rows could not be made");
    CK(cudaStreamSynchronize(s));   // the temporaries are freed on return
    G.valid = true;
    return VRS_OK;
}

vrs_status vrs_range_query(vrs_engine *e, const float *q, int32_t batch, int32_t d,
                           const vrs_pred *pred, float eps, vrs_metric metric, int64_t cap,
                           int64_t *out_offsets, int64_t *out_ids, float *out_dist,
                           int io_on_device, void *stream) {
    NvtxRange nvtx_range("vrs_range_query");
    if (!e || !q || !pred || !out_offsets) return fail(VRS_EINVAL, "NULL argument");
    if (e->n == 0) return fail(VRS_ESTATE, "no vectors loaded");
    if (batch < 1 || batch > 64) return fail(VRS_EINVAL, "batch=%d out of 1..64", batch);
    if (d != e->d) return fail(VRS_EINVAL, "query dimension %d != loaded %d", d, e->d);
    if (metric != VRS_L2 && metric != VRS_IP) return fail(VRS_EINVAL, "bad metric %d", metric);
    if (std::isnan(eps)) return fail(VRS_EINVAL, "eps is NaN");
    if (cap < 0 || (cap > 0 && (!out_ids || !out_dist)))
        return fail(VRS_EINVAL, "cap=%lld needs out_ids and out_dist", (long long)cap);
    if (!e->has[VRS_F32]) return fail(VRS_EINVAL, "range search needs the float32 copy");
    if ((int64_t)batch * e->n * 4 > ((int64_t)256 << 20) || e->ld > 2048)
        return fail(VRS_EINVAL, "the [batch x rows] key matrix must fit 256 MB (and d <= 2048)");
    PredArg p{};
    TRY(check_pred(e, pred, &p));
    DeviceGuard g(e->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (s == nullptr) {
        if (!e->own) CK(cudaStreamCreateWithFlags(&e->own, cudaStreamNonBlocking));
        s = e->own;
    }
    e->marks.clear();
    e->ev_used = 0;
    e->launches = 0;
    e->profiled_last = false;

    // queries on the device, padded to the row stride
    const float *qsrc = q;
    if (!io_on_device) {
        TRY(e->qin.ensure((size_t)batch * d * 4));
        CK(cudaMemcpyAsync(e->qin.p, q, (size_t)batch * d * 4, cudaMemcpyHostToDevice, s));
        qsrc = e->qin.as<const float>();
    }
    {
        const size_t before = e->tau_g.bytes;
        TRY(e->tau_g.ensure((size_t)batch * 8));
        TRY(e->cand_cnt.ensure((size_t)batch * 4));
        if (e->tau_g.bytes != before) {
            CK(cudaMemsetAsync(e->tau_g.p, 0xFF, e->tau_g.bytes, s));
            CK(cudaMemsetAsync(e->cand_cnt.p, 0, e->cand_cnt.bytes, s));
        }
    }
    const float *qdev = qsrc;
    if (e->ld != d) {
        TRY(e->qpad.ensure((size_t)batch * e->ld * 4));
        CK(launch_prep_queries(qsrc, batch, d, e->qpad.as<float>(), e->ld, e->tau_g.as<uint64_t>(),
                               e->cand_cnt.as<int32_t>(), s));
        e->launches += 1;
        qdev = e->qpad.as<const float>();
    }

    // selected ids, then every first-pass key (the GEMV plan's dense-key pass)
    TRY(e->ids.ensure((size_t)e->n * 4));
    TRY(e->count_q.ensure(64));
    CK(cudaMemsetAsync(e->count_q.p, 0, 8, s));
    CK(launch_predicate_ids(attr_arg(e), e->n, p, nullptr, e->ids.as<int32_t>(),
                            e->count_q.as<int64_t>(), e->n_sm, s));
    TRY(e->keys.ensure((size_t)batch * keys_ld(e) * 4));
    TRY(e->cmin.ensure((size_t)batch * cmin_ld(e) * 4));
    const double s_est = estimate_selectivity(e, p);
    const int64_t count = std::min<int64_t>(e->n, (int64_t)std::ceil(s_est * e->n) + 256);
    const int qb = scan_simt_query_block(batch);
    const int nqg = (batch + qb - 1) / qb;
    int G = e->grid_ctas > 0 ? e->grid_ctas : std::max(1, (8 * e->n_sm + nqg - 1) / nqg);
    G = (int)std::min<int64_t>(G, std::max<int64_t>(1, (count + 127) / 128));
    ScanArgs a{};
    a.X = e->x32.p;
    a.x_bf16 = 0;
    a.ld = e->ld;
    a.d = e->d;
    a.xnorm = e->norms.as<const float>();
    a.ids = e->ids.as<const int32_t>();
    a.count_dev = e->count_q.as<const int64_t>();
    a.n_rows = e->n;
    a.Q = qdev;
    a.B = batch;
    a.metric = metric;
    a.kp = 1;
    a.tau_g = e->tau_g.as<uint64_t>();
    a.out_cnt = e->cand_cnt.as<int32_t>();
    a.keys_out = e->keys.as<float>();
    a.keys_ld = keys_ld(e);
    a.chunk_min = e->cmin.as<uint32_t>();
    a.cmin_ld = cmin_ld(e);
    a.err = e->err.as<int32_t>();
    TRY(run_keys_scan(e, a, batch, G, s));
    e->launches += 2;
    if (!e->xn_max_valid) {
        TRY(e->xn_max.ensure(16));
        CK(launch_max_f32(e->norms.as<const float>(), e->n, e->xn_max.as<float>(), s));
        e->launches += 1;
        e->xn_max_valid = true;
    }

    // mark pass: exact scores near and below the bound, counts per query
    RangeArgs r{};
    r.keys = e->keys.as<float>();
    r.keys_ld = keys_ld(e);
    r.chunk_min = e->cmin.as<uint32_t>();
    r.cmin_ld = cmin_ld(e);
    r.ids = e->ids.as<const int32_t>();
    r.count_dev = e->count_q.as<const int64_t>();
    r.X = e->x32.as<const float>();
    r.ld = e->ld;
    r.d = e->d;
    r.Q = qdev;
    r.xn_max = e->xn_max.as<const float>();
    r.B = batch;
    r.metric = metric;
    r.eps = eps;
    TRY(e->rcount.ensure((size_t)batch * 8));
    r.counts = e->rcount.as<int64_t>();
    CK(launch_range_mark(r, s));
    e->launches += 1;
    if (!e->h_rcount) {
        void *h = nullptr;
        CK(cudaMallocHost(&h, 65 * sizeof(int64_t)));
        e->h_rcount = static_cast<int64_t *>(h);
    }
    CK(cudaMemcpyAsync(e->h_rcount, e->rcount.p, (size_t)batch * 8, cudaMemcpyDeviceToHost, s));
    TRY(check_device_error(e, s));   // synchronises the stream
    out_offsets[0] = 0;
    for (int i = 0; i < batch; ++i) out_offsets[i + 1] = out_offsets[i] + e->h_rcount[i];
    const int64_t total = out_offsets[batch];
    // the selected-row count goes back to zero for the next query (the
    // top-k merge leaves it so too)
    if (total > cap || total == 0) {
        CK(cudaMemsetAsync(e->count_q.p, 0, 8, s));
        if (total == 0) return VRS_OK;
        return fail(VRS_ESIZE, "%lld results, capacity %lld", (long long)total, (long long)cap);
    }

    // write pass at the offsets
    TRY(e->roff.ensure((size_t)(batch + 1) * 8));
    CK(cudaMemcpyAsync(e->roff.p, out_offsets, (size_t)(batch + 1) * 8, cudaMemcpyHostToDevice, s));
    r.offsets = e->roff.as<const int64_t>();
    if (io_on_device) {
        r.out_ids = out_ids;
        r.out_dist = out_dist;
    } else {
        TRY(e->rids.ensure((size_t)total * 8));
        TRY(e->rdist.ensure((size_t)total * 4));
        r.out_ids = e->rids.as<int64_t>();
        r.out_dist = e->rdist.as<float>();
    }
    CK(launch_range_write(r, s));
    e->launches += 1;
    CK(cudaMemsetAsync(e->count_q.p, 0, 8, s));
    if (!io_on_device) {
        CK(cudaMemcpyAsync(out_ids, r.out_ids, (size_t)total * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(out_dist, r.out_dist, (size_t)total * 4, cudaMemcpyDeviceToHost, s));
        TRY(check_device_error(e, s));
    }
    return VRS_OK;
}

vrs_status vrs_query_dnf(vrs_engine *e, const float *q, int32_t batch, int32_t d,
                         const vrs_pred *conj, int32_t n_conj, int32_t k, vrs_metric metric,
                         vrs_dtype compute, int64_t *out_ids, float *out_dist, int io_on_device,
                         void *stream) {
    NvtxRange nvtx_range("vrs_query_dnf");
    if (!e || !q || !conj || !out_ids || !out_dist) return fail(VRS_EINVAL, "NULL argument");
    if (e->n == 0) return fail(VRS_ESTATE, "no vectors loaded");
    if (batch < 1) return fail(VRS_EINVAL, "batch=%d must be >= 1", batch);
    if (d != e->d) return fail(VRS_EINVAL, "query dimension %d != loaded %d", d, e->d);
    if (k < 1 || k > kMaxK) return fail(VRS_EINVAL, "k=%d out of 1..%d", k, kMaxK);
    if (n_conj < 1 || (int64_t)n_conj * k > union_max_entries())
        return fail(VRS_EINVAL, "n_conj=%d: need 1 <= n_conj and n_conj * k <= %d", n_conj,
                    union_max_entries());
    if (metric != VRS_L2 && metric != VRS_IP) return fail(VRS_EINVAL, "bad metric %d", metric);
    if (compute < VRS_F32 || compute > VRS_FP8E4M3 || !e->has[compute])
        return fail(VRS_EINVAL, "compute encoding %d is not resident", compute);
    std::vector<PredArg> pa((size_t)n_conj);
    for (int i = 0; i < n_conj; ++i) TRY(check_pred(e, &conj[i], &pa[(size_t)i]));
    DeviceGuard g(e->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (!io_on_device && s == nullptr) {
        if (!e->own) CK(cudaStreamCreateWithFlags(&e->own, cudaStreamNonBlocking));
        s = e->own;
    }
    e->marks.clear();
    e->ev_used = 0;
    e->launches = 0;
    for (auto &c : e->cert_count) c = 0;
    e->cert_lazy_n = 0;
    e->profiled_last = false;
    const float *qdev = q;
    if (!io_on_device) {
        TRY(e->qin.ensure((size_t)batch * d * 4));
        CK(cudaMemcpyAsync(e->qin.p, q, (size_t)batch * d * 4, cudaMemcpyHostToDevice, s));
        qdev = e->qin.as<const float>();
    }
    {
        const size_t before = e->tau_g.bytes;
        TRY(e->tau_g.ensure((size_t)batch * 8));
        TRY(e->cand_cnt.ensure((size_t)batch * 4));
        if (e->tau_g.bytes != before) {
            CK(cudaMemsetAsync(e->tau_g.p, 0xFF, e->tau_g.bytes, s));
            CK(cudaMemsetAsync(e->cand_cnt.p, 0, e->cand_cnt.bytes, s));
        }
    }
    // the top-k of each conjunction's rows, then the k best of their union
    const int64_t stride = (int64_t)batch * k;
    TRY(e->uids.ensure((size_t)n_conj * stride * 8));
    TRY(e->udist.ensure((size_t)n_conj * stride * 4));
    int64_t launches = 0;
    for (int i = 0; i < n_conj; ++i) {
        e->launches = 0;
        TRY(query_shared_exact(e, qdev, batch, pa[(size_t)i], nullptr, k, k, metric, compute,
                               e->uids.as<int64_t>() + i * stride,
                               e->udist.as<float>() + i * stride, s));
        launches += e->launches;
    }
    UnionArgs u{};
    u.ids = e->uids.as<const int64_t>();
    u.dist = e->udist.as<const float>();
    u.list_stride = stride;
    u.n_lists = n_conj;
    u.k = k;
    u.B = batch;
    u.metric = metric;
    if (io_on_device) {
        u.out_ids = out_ids;
        u.out_dist = out_dist;
    } else {
        TRY(e->oid.ensure((size_t)stride * 8));
        TRY(e->odist.ensure((size_t)stride * 4));
        u.out_ids = e->oid.as<int64_t>();
        u.out_dist = e->odist.as<float>();
    }
    CK(launch_union_topk(u, s));
    e->launches = launches + 1;
    if (!io_on_device) {
        CK(cudaMemcpyAsync(out_ids, u.out_ids, (size_t)stride * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(out_dist, u.out_dist, (size_t)stride * 4, cudaMemcpyDeviceToHost, s));
        TRY(check_device_error(e, s));
    }
    return VRS_OK;
}

vrs_status vrs_join_topk(vrs_engine *e, const float *qrel, int64_t m, int32_t d,
                         const int32_t *qattrs, int32_t q_cols, const vrs_pred *qpred,
                         const vrs_pred *rpred, int32_t k, vrs_metric metric, vrs_dtype compute,
                         int64_t cap, int64_t *out_nq, int64_t *out_qids, int64_t *out_ids,
                         float *out_dist, int io_on_device, void *stream) {
    NvtxRange nvtx_range("vrs_join_topk");
    if (!e || !qrel || !qpred || !rpred || !out_nq) return fail(VRS_EINVAL, "NULL argument");
    if (e->n == 0) return fail(VRS_ESTATE, "no vectors loaded");
    if (m < 1 || m > 0x7fffffffLL) return fail(VRS_EINVAL, "m=%lld out of range", (long long)m);
    if (d != e->d) return fail(VRS_EINVAL, "query dimension %d != loaded %d", d, e->d);
    if (q_cols < 0 || q_cols > kMaxCols || (q_cols > 0 && !qattrs))
        return fail(VRS_EINVAL, "q_cols=%d (with qattrs) out of 0..%d", q_cols, kMaxCols);
    if (k < 1 || k > kMaxK) return fail(VRS_EINVAL, "k=%d out of 1..%d", k, kMaxK);
    if (metric != VRS_L2 && metric != VRS_IP) return fail(VRS_EINVAL, "bad metric %d", metric);
    if (compute < VRS_F32 || compute > VRS_FP8E4M3 || !e->has[compute])
        return fail(VRS_EINVAL, "compute encoding %d is not resident", compute);
    if (cap < 0 || (cap > 0 && (!out_qids || !out_ids || !out_dist)))
        return fail(VRS_EINVAL, "cap=%lld needs out_qids, out_ids and out_dist", (long long)cap);
    PredArg rp{};
    TRY(check_pred(e, rpred, &rp));
    PredArg qp{};
    if (qpred->n_terms < 0 || qpred->n_terms > kMaxTerms || (qpred->n_terms && !qpred->terms))
        return fail(VRS_EINVAL, "bad query-relation predicate");
    qp.n_terms = qpred->n_terms;
    for (int t = 0; t < qp.n_terms; ++t) {
        const vrs_range &r = qpred->terms[t];
        if (r.col < 0 || r.col >= q_cols)
            return fail(VRS_EINVAL, "query-relation predicate column %d out of 0..%d", r.col, q_cols - 1);
        qp.col[t] = r.col;
        qp.lo[t] = r.lo;
        qp.hi[t] = r.hi;
    }
    DeviceGuard g(e->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (s == nullptr) {
        if (!e->own) CK(cudaStreamCreateWithFlags(&e->own, cudaStreamNonBlocking));
        s = e->own;
    }
    e->marks.clear();
    e->ev_used = 0;
    e->launches = 0;
    for (auto &c : e->cert_count) c = 0;
    e->cert_lazy_n = 0;
    e->profiled_last = false;
    const cudaMemcpyKind kind = io_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;

    // the query relation on the device; its attribute columns 16-byte aligned
    const float *qdev = qrel;
    if (!io_on_device) {
        TRY(e->jq.ensure((size_t)m * d * 4));
        CK(cudaMemcpyAsync(e->jq.p, qrel, (size_t)m * d * 4, cudaMemcpyHostToDevice, s));
        qdev = e->jq.as<const float>();
    }
    const int64_t m4 = (m + 3) & ~(int64_t)3;
    AttrArg qa{};
    if (q_cols > 0) {
        TRY(e->jqa.ensure((size_t)q_cols * m4 * 4 + 16));
        CK(cudaMemcpy2DAsync(e->jqa.p, (size_t)m4 * 4, qattrs, (size_t)m * 4, (size_t)m * 4,
                             (size_t)q_cols, kind, s));
        for (int c = 0; c < q_cols; ++c) qa.col[c] = e->jqa.as<const int32_t>() + (int64_t)c * m4;
    }
    // sigma over the query relation: bitmap, tile offsets, ascending ids
    const int64_t nt = n_tiles(m);
    TRY(e->jbm.ensure((size_t)((m + 31) / 32) * 4 + 16));
    TRY(e->jtc.ensure((size_t)nt * 4));
    TRY(e->jto.ensure((size_t)nt * 8));
    TRY(e->jcnt.ensure(64));
    TRY(e->jqids.ensure((size_t)m * 4));
    CK(launch_predicate(qa, m, qp, e->jbm.as<uint32_t>(), e->jtc.as<int32_t>(), s));
    CK(launch_tile_scan(e->jtc.as<int32_t>(), nt, e->jto.as<int64_t>(), e->jcnt.as<int64_t>(), s));
    CK(launch_compact(e->jbm.as<uint32_t>(), m, e->jto.as<int64_t>(), e->jqids.as<int32_t>(), s));
    CK(cudaMemcpyAsync(e->h_count, e->jcnt.p, 8, cudaMemcpyDeviceToHost, s));
    TRY(check_device_error(e, s));   // synchronises the stream
    const int64_t nq = e->h_count[0];
    *out_nq = nq;
    if (nq > cap) return fail(VRS_ESIZE, "%lld query rows selected, capacity %lld", (long long)nq, (long long)cap);
    if (nq == 0) return VRS_OK;

    // the selected queries, gathered; then the filtered top-k per batch of
    // up to kJoinBatch of them through the ordinary query path
    TRY(e->jgq.ensure((size_t)nq * d * 4));
    CK(launch_gather_rows_f32(qdev, d, e->jqids.as<const int32_t>(), nq, e->jgq.as<float>(), s));
    int64_t *oid = out_ids;
    float *odist = out_dist;
    if (!io_on_device) {
        TRY(e->joid.ensure((size_t)nq * k * 8));
        TRY(e->jodist.ensure((size_t)nq * k * 4));
        oid = e->joid.as<int64_t>();
        odist = e->jodist.as<float>();
    }
    constexpr int64_t kJoinBatch = 4096;
    {
        const int64_t bmax = std::min(nq, kJoinBatch);
        const size_t before = e->tau_g.bytes;
        TRY(e->tau_g.ensure((size_t)bmax * 8));
        TRY(e->cand_cnt.ensure((size_t)bmax * 4));
        if (e->tau_g.bytes != before) {
            CK(cudaMemsetAsync(e->tau_g.p, 0xFF, e->tau_g.bytes, s));
            CK(cudaMemsetAsync(e->cand_cnt.p, 0, e->cand_cnt.bytes, s));
        }
    }
    const int64_t launches0 = e->launches + 4;
    int64_t launches = launches0;
    for (int64_t off = 0; off < nq; off += kJoinBatch) {
        const int32_t bsz = (int32_t)std::min(kJoinBatch, nq - off);
        e->launches = 0;
        TRY(query_shared_exact(e, e->jgq.as<const float>() + off * d, bsz, rp, nullptr, k, k,
                               metric, compute, oid + off * k, odist + off * k, s));
        launches += e->launches;
    }
    e->launches = launches;
    std::vector<int32_t> qids((size_t)nq);
    CK(cudaMemcpyAsync(qids.data(), e->jqids.p, (size_t)nq * 4, cudaMemcpyDeviceToHost, s));
    if (!io_on_device) {
        CK(cudaMemcpyAsync(out_ids, oid, (size_t)nq * k * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(out_dist, odist, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, s));
    }
    TRY(check_device_error(e, s));
    for (int64_t i = 0; i < nq; ++i) out_qids[i] = qids[(size_t)i];
    return VRS_OK;
}

vrs_status vrs_eval_predicate(vrs_engine *e, const vrs_pred *pred, uint32_t *bitmap_out,
                              int64_t *count_out, int out_on_device, void *stream) {
    if (!e || !count_out) return fail(VRS_EINVAL, "engine or count_out is NULL");
    if (e->n == 0) return fail(VRS_ESTATE, "no vectors loaded");
    DeviceGuard g(e->device);
    PredArg p;
    TRY(check_pred(e, pred, &p));
    cudaStream_t s = (cudaStream_t)stream;
    TRY(run_filter(e, p, s));
    if (bitmap_out)
        CK(cudaMemcpyAsync(bitmap_out, e->bitmap.p, (size_t)((e->n + 31) / 32) * 4,
                           out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    return read_count(e, s, count_out);
}

vrs_status vrs_probe_gather(const void *rows, int64_t n_rows, int64_t row_bytes, const int32_t *ids,
                            int64_t m, float *out, void *stream) {
    if (!rows || !out || (m > 0 && !ids)) return fail(VRS_EINVAL, "NULL argument");
    if (m < 0 || n_rows < 0 || row_bytes < 16 || row_bytes % 16 ||
        reinterpret_cast<uintptr_t>(rows) % 16)
        return fail(VRS_EINVAL, "rows must be 16-byte aligned, row_bytes a positive multiple of 16");
    int dev = 0, n_sm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    CK(launch_gather_probe(rows, n_rows, row_bytes, ids, m, out, n_sm, (cudaStream_t)stream));
    return VRS_OK;
}

vrs_status vrs_select_ids(vrs_engine *e, const vrs_pred *pred, int32_t *ids_out,
                          int64_t *count_out, int out_on_device, void *stream) {
    if (!e || !count_out || !ids_out) return fail(VRS_EINVAL, "NULL argument");
    if (e->n == 0) return fail(VRS_ESTATE, "no vectors loaded");
    DeviceGuard g(e->device);
    PredArg p;
    TRY(check_pred(e, pred, &p));
    cudaStream_t s = (cudaStream_t)stream;
    TRY(run_filter(e, p, s));
    TRY(run_compact(e, s));
    TRY(read_count(e, s, count_out));
    if (*count_out > 0)
        CK(cudaMemcpyAsync(ids_out, e->ids.p, (size_t)*count_out * 4,
                           out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return VRS_OK;
}

vrs_status vrs_get_norms(vrs_engine *e, float *out, int out_on_device, void *stream) {
    if (!e || !out) return fail(VRS_EINVAL, "NULL argument");
    if (e->n == 0) return fail(VRS_ESTATE, "no vectors loaded");
    DeviceGuard g(e->device);
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(out, e->norms.p, (size_t)e->n * 4,
                       out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return VRS_OK;
}

vrs_status vrs_get_encoded(vrs_engine *e, vrs_dtype dt, void *codes_out, float *scale_out,
                           int out_on_device, void *stream) {
    if (!e || !codes_out) return fail(VRS_EINVAL, "NULL argument");
    if (dt < VRS_F32 || dt > VRS_FP8E4M3) return fail(VRS_EINVAL, "bad dtype %d", dt);
    if (e->n == 0 || !e->has[dt]) return fail(VRS_ESTATE, "encoding %d not resident", dt);
    DeviceGuard g(e->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t esz = dt == VRS_F32 ? 4 : dt == VRS_BF16 ? 2 : 1;
    const void *src = dt == VRS_F32 ? e->x32.p : dt == VRS_BF16 ? e->xb.p : e->x8.p;
    cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpy2DAsync(codes_out, (size_t)e->d * esz, src, (size_t)e->ld * esz,
                         (size_t)e->d * esz, (size_t)e->n, kind, s));
    if (dt == VRS_FP8E4M3 && scale_out)
        CK(cudaMemcpyAsync(scale_out, e->s8.p, (size_t)e->n * 4, kind, s));
    CK(cudaStreamSynchronize(s));
    return VRS_OK;
}

vrs_status vrs_query(vrs_engine *e, const float *q, int32_t batch, int32_t d,
                     const vrs_pred *preds, int32_t n_preds, const int32_t *k, int32_t n_k,
                     int32_t k_max, vrs_metric metric, vrs_dtype compute, int64_t *out_ids,
                     float *out_dist, int io_on_device, void *stream) {
    NvtxRange nvtx_range("vrs_query");
    if (!e || !q || !preds || !k || !out_ids || !out_dist)
        return fail(VRS_EINVAL, "NULL argument");
    if (e->n == 0) return fail(VRS_ESTATE, "no vectors loaded");
    if (batch < 1) return fail(VRS_EINVAL, "batch=%d must be >= 1", batch);
    if (d != e->d) return fail(VRS_EINVAL, "query dimension %d != loaded %d", d, e->d);
    if (n_preds != 1 && n_preds != batch)
        return fail(VRS_EINVAL, "n_preds=%d must be 1 or batch=%d", n_preds, batch);
    if (n_k != 1 && n_k != batch) return fail(VRS_EINVAL, "n_k=%d must be 1 or batch", n_k);
    if (k_max < 1 || k_max > kMaxK) return fail(VRS_EINVAL, "k_max=%d out of 1..%d", k_max, kMaxK);
    for (int i = 0; i < n_k; ++i)
        if (k[i] < 0 || k[i] > k_max) return fail(VRS_EINVAL, "k[%d]=%d out of 0..k_max", i, k[i]);
    if (metric != VRS_L2 && metric != VRS_IP) return fail(VRS_EINVAL, "bad metric %d", metric);
    if (compute < VRS_F32 || compute > VRS_FP8E4M3 || !e->has[compute])
        return fail(VRS_EINVAL, "compute encoding %d is not resident", compute);
    std::vector<PredArg> pa(n_preds);
    for (int i = 0; i < n_preds; ++i) TRY(check_pred(e, &preds[i], &pa[i]));
    DeviceGuard g(e->device);
    cudaStream_t s = (cudaStream_t)stream;
    // a host-buffer query is synchronous; without a caller stream it runs on
    // the engine's own stream, so the captured-graph forms apply to it too
    if (!io_on_device && s == nullptr) {
        if (!e->own) CK(cudaStreamCreateWithFlags(&e->own, cudaStreamNonBlocking));
        s = e->own;
    }
    e->marks.clear();
    e->ev_used = 0;
    e->launches = 0;
    for (auto &c : e->cert_count) c = 0;
    e->cert_lazy_n = 0;
    e->profiled_last = e->profile;

    // queries on the device.  Page-locked host buffers with one shared
    // predicate: the captured GEMV form copies them inside its graph.
    // (a page-locked host buffer's device address, or NULL)
    auto pinned = [](const void *ptr) -> void * {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return at.type == cudaMemoryTypeHost ? (at.devicePointer ? at.devicePointer : (void *)ptr)
                                             : nullptr;
    };
    void *q_dev_map = nullptr, *ids_dev_map = nullptr, *dist_dev_map = nullptr;
    const bool pinned_io = !io_on_device && n_preds == 1 && (q_dev_map = pinned(q)) &&
                           (ids_dev_map = pinned(out_ids)) && (dist_dev_map = pinned(out_dist));
    e->io_q_host = nullptr;
    e->io_ids_host = nullptr;
    e->io_dist_host = nullptr;
    e->io_q_dev = pinned_io ? static_cast<const float *>(q_dev_map) : nullptr;
    e->io_ids_dev = pinned_io ? static_cast<int64_t *>(ids_dev_map) : nullptr;
    e->io_dist_dev = pinned_io ? static_cast<float *>(dist_dev_map) : nullptr;
    e->io_out_done = false;
    const float *qsrc = q;
    if (!io_on_device) {
        TRY(e->qin.ensure((size_t)batch * d * 4));
        if (pinned_io) {
            e->io_q_host = q;
            e->io_q_bytes = (size_t)batch * d * 4;
        } else {
            CK(cudaMemcpyAsync(e->qin.p, q, (size_t)batch * d * 4, cudaMemcpyHostToDevice, s));
        }
        qsrc = e->qin.as<const float>();
    }
    // per-query search state: kept cleared between queries by the merge
    // kernel; set here whenever the buffers are (re)allocated
    {
        const size_t before = e->tau_g.bytes;
        TRY(e->tau_g.ensure((size_t)batch * 8));
        TRY(e->cand_cnt.ensure((size_t)batch * 4));
        if (e->tau_g.bytes != before) {
            CK(cudaMemsetAsync(e->tau_g.p, 0xFF, e->tau_g.bytes, s));
            CK(cudaMemsetAsync(e->cand_cnt.p, 0, e->cand_cnt.bytes, s));
        }
    }

    int64_t *oid = out_ids;
    float *odist = out_dist;
    if (!io_on_device) {
        TRY(e->oid.ensure((size_t)batch * k_max * 8));
        TRY(e->odist.ensure((size_t)batch * k_max * 4));
        oid = e->oid.as<int64_t>();
        odist = e->odist.as<float>();
    }

    if (n_preds == 1) {
        const int32_t *kd = nullptr;
        int32_t ks = k[0];
        if (n_k == batch) {
            bool same = true;
            for (int i = 1; i < n_k; ++i) same = same && k[i] == k[0];
            if (!same) {
                TRY(e->staging.ensure((size_t)batch * 4));
                CK(cudaMemcpyAsync(e->staging.p, k, (size_t)batch * 4, cudaMemcpyHostToDevice, s));
                kd = e->staging.as<const int32_t>();
            }
        }
        if (pinned_io) {
            e->io_ids_host = out_ids;
            e->io_dist_host = out_dist;
            e->io_out_n = (size_t)batch * k_max;
        }
        const vrs_status st = query_shared_exact(e, qsrc, batch, pa[0], kd, ks, k_max, metric,
                                                 compute, oid, odist, s);
        e->io_q_host = nullptr;
        e->io_ids_host = nullptr;
        e->io_dist_host = nullptr;
        TRY(st);
    } else {
        TRY(e->cflag.ensure((size_t)batch * 4));
        TRY(e->cdup.ensure((size_t)batch * 4));
        e->cur_cflag = e->cflag.as<int32_t>();
        e->cur_cdup = e->cdup.as<float>();
        e->rerank_merge = false;
        bool done = false;
        const bool any_plan = e->plan_forced == VRS_PLAN_AUTO || e->plan_forced == VRS_PLAN_CELLS;
        if (e->batched && any_plan && cells_eligible(e, pa, compute)) {
            // the dense-key merge certifies every query itself
            TRY(query_cells(e, qsrc, batch, pa, k, n_k, k_max, metric, oid, odist, s));
            done = true;
        }
        if (!done && e->batched && compute != VRS_F32 && e->plan_forced != VRS_PLAN_GEMV &&
            e->plan_forced != VRS_PLAN_COMPACT_GEMM && e->plan_forced != VRS_PLAN_CELLS) {
            TRY(query_batched(e, qsrc, batch, pa, k, n_k, k_max, metric, compute, oid, odist, s,
                              &done));
            if (done) e->rerank_merge = true;   // the batched merge flags its queries
        }
        // otherwise one predicate per query: one pass per query
        for (int i = 0; i < batch && !done; ++i) {
            int32_t ki = n_k == 1 ? k[0] : k[i];
            e->cur_cflag = e->cflag.as<int32_t>() + i;
            e->cur_cdup = e->cdup.as<float>() + i;
            TRY(query_shared(e, qsrc + (int64_t)i * d, e->tau_g.as<uint64_t>() + i,
                             e->cand_cnt.as<int32_t>() + i, 1, pa[i], nullptr, ki, k_max, metric,
                             compute, oid + (int64_t)i * k_max, odist + (int64_t)i * k_max, s));
        }
        e->cur_cflag = e->cflag.as<int32_t>();
        e->cur_cdup = e->cdup.as<float>();
        // the per-query k on the device for the re-runs (a self-certified
        // pass needs none)
        const int32_t *kd = nullptr;
        if (n_k == batch && e->rerank_merge) {
            TRY(e->staging.ensure((size_t)batch * 4));
            CK(cudaMemcpyAsync(e->staging.p, k, (size_t)batch * 4, cudaMemcpyHostToDevice, s));
            kd = e->staging.as<const int32_t>();
        }
        TRY(certify_batch(e, qsrc, batch, nullptr, &pa, kd, k[0], k_max, metric, compute, oid,
                          odist, s));
    }
    if (!io_on_device) {
        if (e->io_out_done) {   // the graph downloaded the results and the error word
            e->io_out_done = false;
            CK(cudaStreamSynchronize(s));
            if (*e->h_err) TRY(check_device_error(e, s));
            return VRS_OK;
        }
        CK(cudaMemcpyAsync(out_ids, oid, (size_t)batch * k_max * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(out_dist, odist, (size_t)batch * k_max * 4, cudaMemcpyDeviceToHost, s));
        TRY(check_device_error(e, s));
    }
    return VRS_OK;
}

vrs_status vrs_merge_shards(const int64_t *ids, const float *dist, int32_t n_shards,
                            int32_t batch, int32_t k, const int64_t *row_offset,
                            vrs_metric metric, int64_t *out_ids, float *out_dist,
                            int io_on_device, void *stream) {
    NvtxRange nvtx_range("vrs_merge_shards");
    if (!ids || !dist || !row_offset || !out_ids || !out_dist)
        return fail(VRS_EINVAL, "NULL argument");
    if (n_shards < 1 || n_shards > kMaxLists)
        return fail(VRS_EINVAL, "n_shards=%d out of 1..%d", n_shards, kMaxLists);
    if (batch < 1) return fail(VRS_EINVAL, "batch=%d must be >= 1", batch);
    if (k < 1 || k > kMaxK || (int64_t)n_shards * k > union_max_entries())
        return fail(VRS_EINVAL, "k=%d: need 1 <= k <= %d and n_shards * k <= %d", k, kMaxK,
                    union_max_entries());
    if (metric != VRS_L2 && metric != VRS_IP) return fail(VRS_EINVAL, "bad metric %d", metric);
    ListOffsets off{};
    off.n = n_shards;
    for (int i = 0; i < n_shards; ++i) {
        if (row_offset[i] < 0 || row_offset[i] > INT32_MAX)
            return fail(VRS_EINVAL, "row_offset[%d]=%lld out of 0..2^31-1", i,
                        (long long)row_offset[i]);
        off.v[i] = row_offset[i];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t m = (size_t)n_shards * batch * k, mo = (size_t)batch * k;
    UnionArgs u{};
    u.list_stride = (int64_t)batch * k;
    u.n_lists = n_shards;
    u.k = k;
    u.B = batch;
    u.metric = metric;
    if (io_on_device) {
        u.ids = ids;
        u.dist = dist;
        u.out_ids = out_ids;
        u.out_dist = out_dist;
        CK(launch_union_topk(u, s, &off));
        return VRS_OK;
    }
    // host buffers: staged through device memory owned by this call
    void *buf = nullptr;
    CK(cudaMalloc(&buf, m * 12 + mo * 12));
    int64_t *di = static_cast<int64_t *>(buf);
    int64_t *doi = di + m;
    float *dd = reinterpret_cast<float *>(doi + mo);
    float *dod = dd + m;
    u.ids = di;
    u.dist = dd;
    u.out_ids = doi;
    u.out_dist = dod;
    cudaError_t ce = cudaMemcpyAsync(di, ids, m * 8, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(dd, dist, m * 4, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = launch_union_topk(u, s, &off);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(out_ids, doi, mo * 8, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(out_dist, dod, mo * 4, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    cudaFree(buf);
    if (ce != cudaSuccess) return fail(VRS_ECUDA, "shard merge failed: %s", cudaGetErrorString(ce));
    return VRS_OK;
}

vrs_status vrs_last_cert(vrs_engine *e, int64_t *counts) {
    if (!e || !counts) return fail(VRS_EINVAL, "NULL argument");
    DeviceGuard g(e->device);
    TRY(flush_cert(e));
    for (int i = 0; i < 4; ++i) counts[i] = e->cert_count[i];
    return VRS_OK;
}

float vrs_cert_bound(int32_t kind, int32_t d, vrs_metric metric, float qnorm, float qres,
                     float xmax, float xres) {
    if (kind < VRS_CERT_FFMA || kind > VRS_CERT_E4M3 || d < 1 ||
        (metric != VRS_L2 && metric != VRS_IP))
        return -1.0f;
    CertArgs c{};
    c.A = xmax;
    c.Rx = xres;
    c.d = d;
    c.P = kind == VRS_CERT_TF32X3   ? cert_P_tf32x3(d)
          : kind == VRS_CERT_BF16X3 ? cert_P_bf16x3(d)
          : kind == VRS_CERT_BF16   ? cert_P_bf16(d)
          : kind == VRS_CERT_E4M3   ? cert_P_e4m3(d)
                                    : cert_P_ffma(d);
    return cert_bound(qnorm, qres, c, (int)metric);
}

vrs_status vrs_set_plan(vrs_engine *e, int plan) {
    if (!e) return fail(VRS_EINVAL, "engine is NULL");
    if (plan < VRS_PLAN_AUTO || plan > VRS_PLAN_CELLS) return fail(VRS_EINVAL, "bad plan %d", plan);
    e->plan_forced = plan;
    return VRS_OK;
}

vrs_status vrs_last_plan(vrs_engine *e, int *plan) {
    if (!e || !plan) return fail(VRS_EINVAL, "NULL argument");
    *plan = e->last_plan;
    return VRS_OK;
}

vrs_status vrs_set_option(vrs_engine *e, int key, int64_t value) {
    if (!e) return fail(VRS_EINVAL, "engine is NULL");
    switch (key) {
        case VRS_OPT_KPRIME_FACTOR:
            if (value < 0 || value > 64) return fail(VRS_EINVAL, "k' factor %lld out of 0..64", (long long)value);
            e->kprime_factor = (int)value;
            return VRS_OK;
        case VRS_OPT_RERANK:
            e->rerank = value != 0;
            return VRS_OK;
        case VRS_OPT_PROFILE:
            e->profile = value != 0;
            return VRS_OK;
        case VRS_OPT_FUSED_SCAN:
            e->fused_gemv = value != 0;
            return VRS_OK;
        case VRS_OPT_BATCHED:
            e->batched = value != 0;
            return VRS_OK;
        case VRS_OPT_GRAPH:
            e->use_graph = value != 0;
            return VRS_OK;
        case VRS_OPT_TMA:
            e->tma = value != 0;
            return VRS_OK;
        case VRS_OPT_DENSE_KEYS:
            e->dense_keys = value != 0;
            return VRS_OK;
        case VRS_OPT_STAGED_SCAN:
            e->staged_scan = value != 0;
            return VRS_OK;
        case VRS_OPT_TENSOR_GEMV:
            e->tensor_gemv = value != 0;
            return VRS_OK;
        case VRS_OPT_SEED_BOUND:
            e->seed_bound = value != 0;
            return VRS_OK;
        case VRS_OPT_PAIR_COPY:
            e->pair_copy = value != 0;
            return VRS_OK;
        case VRS_OPT_WAIT_TEST:
            e->wait_test = value != 0;
            return VRS_OK;
        case VRS_OPT_CERT_SAMPLE:
            e->cert_sample = value != 0;
            return VRS_OK;
        case VRS_OPT_CELL_PLAN:
            e->cell_plan = value != 0;
            return VRS_OK;
        case VRS_OPT_ZERO_COPY:
            e->zero_copy = value != 0;
            return VRS_OK;
        case VRS_OPT_SELECT_CAP:
            if (value < 0 || value > ((int64_t)1 << 30)) return fail(VRS_EINVAL, "capacity %lld out of range", (long long)value);
            e->select_cap = value;
            return VRS_OK;
        case VRS_OPT_GRID_CTAS:
            if (value < 0 || value > 65535) return fail(VRS_EINVAL, "grid %lld out of range", (long long)value);
            e->grid_ctas = (int)value;
            return VRS_OK;
        default:
            return fail(VRS_EINVAL, "unknown option %d", key);
    }
}

vrs_status vrs_last_profile(vrs_engine *e, float *stage_ms, int32_t *launches,
                            int64_t *selected) {
    if (!e) return fail(VRS_EINVAL, "engine is NULL");
    if (launches) *launches = e->launches;
    if (selected) {
        *selected = e->last_count;
        (void)selected;
    }
    if (!stage_ms) return VRS_OK;
    if (!e->profiled_last) return fail(VRS_ESTATE, "the last query ran without VRS_OPT_PROFILE");
    DeviceGuard g(e->device);
    TRY(check_device_error(e, nullptr));
    for (int i = 0; i < VRS_N_STAGES; ++i) stage_ms[i] = 0.0f;
    for (const auto &m : e->marks) {
        CK(cudaEventSynchronize(m.b));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, m.a, m.b));
        stage_ms[m.stage] += ms;
    }
    return VRS_OK;
}

vrs_status vrs_planner_load(vrs_engine *e, const char *path) {
    if (!e) return fail(VRS_EINVAL, "engine is NULL");
    if (!path) {
        e->planner = false;
        return VRS_OK;
    }
    FILE *f = fopen(path, "rb");
    if (!f) return fail(VRS_EIO, "planner file %s cannot be opened; fixed rule kept", path);
    std::vector<unsigned char> buf;
    unsigned char tmp[4096];
    size_t got;
    while ((got = fread(tmp, 1, sizeof tmp, f)) > 0) buf.insert(buf.end(), tmp, tmp + got);
    fclose(f);
    const size_t body = 8 + 4 + 4 + 12 * 4 + 2 * 4 + (size_t)kPlNP * 4;
    if (buf.size() != body + 8) return fail(VRS_EIO, "planner file %s: wrong size; fixed rule kept", path);
    if (memcmp(buf.data(), "VRSPLAN1", 8) != 0)
        return fail(VRS_EIO, "planner file %s: bad magic; fixed rule kept", path);
    uint32_t ver, np;
    memcpy(&ver, buf.data() + 8, 4);
    memcpy(&np, buf.data() + 12, 4);
    if (ver != 1 || np != (uint32_t)kPlNP)
        return fail(VRS_EIO, "planner file %s: unsupported version or size; fixed rule kept", path);
    uint64_t ck;
    memcpy(&ck, buf.data() + body, 8);
    if (ck != fnv1a(buf.data(), body))
        return fail(VRS_EIO, "planner file %s: checksum mismatch; fixed rule kept", path);
    const unsigned char *p = buf.data() + 16;
    memcpy(e->pl_fmean, p, 24);
    memcpy(e->pl_fstd, p + 24, 24);
    memcpy(&e->pl_omean, p + 48, 4);
    memcpy(&e->pl_ostd, p + 52, 4);
    e->pl_params.resize(kPlNP);
    memcpy(e->pl_params.data(), p + 56, (size_t)kPlNP * 4);
    for (int c = 0; c < 6; ++c)
        if (!(e->pl_fstd[c] > 0.0f)) e->pl_fstd[c] = 1.0f;
    // bf16 inference: weights rounded once (biases stay float32)
    for (int i = 0; i < kPlNP; ++i) {
        const bool bias = (i >= 384 && i < 448) || (i >= 4544 && i < 4608) || i >= 4800;
        if (!bias) e->pl_params[i] = bf16r(e->pl_params[i]);
    }
    e->planner = true;
    return VRS_OK;
}

}  // extern "C"
