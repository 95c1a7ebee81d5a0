// knn_capi.cu -- the C ABI declared in include/knn.h: handles, reference sets
// (shareable between handles), workspace and the orchestration of one search
// (select -> finalize -> fallback), all enqueued on one CUDA stream.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <vector>
#include <new>
#include <string>

#include "../../include/knn.h"
#include "knn_batch.cuh"
#include "knn_internal.cuh"

using namespace knn;

namespace {

constexpr int kMaxStages = 8;
// A host-buffer search runs in up to kMaxParts parts of at least
// kPartMinQueries queries each (four parts measured no faster than two at
// n = 38400: 62.2 against 62.3-62.4 million queries/s end to end).
constexpr int kMaxParts = 2;
constexpr int64_t kPartMinQueries = 4096;

// Device counters owned by a handle.
struct Counters {
    int32_t fallback_count;                 // queued queries of the current search
    int32_t fallback_part[kMaxParts - 1];   // the same, parts after the first of a host-buffer search
    int32_t error_flag;                     // set by a kernel whose bounded wait gave up
    unsigned long long recheck_total;       // re-checked near-tie candidates
    unsigned long long fallback_total;      // queries finished by the fallback
    unsigned long long fallback_reason[4];  // short list, overflow, wide cut, uncertified
};

// A reference set on the device, shared by every handle created from it with
// knn_create_shared; freed with the last of them.
struct RefSet {
    int device = 0;
    float* R = nullptr;
    int64_t m = 0;
    int32_t d = 0;
    float* r_norms = nullptr;     // ||r||^2 in float32 (padded to whole tiles)
    void* R_lp = nullptr;         // bf16 / tf32 operand copy
    int32_t kp = 0;               // padded row length of R_lp
    int lp_prec = 0;              // 0: none, kTF32, kBF16
    uint32_t* rmax2 = nullptr;    // device: largest ||r||^2 (float bits)
    ~RefSet() {
        cudaSetDevice(device);
        if (R) cudaFree(R);
        if (r_norms) cudaFree(r_norms);
        if (R_lp) cudaFree(R_lp);
        if (rmax2) cudaFree(rmax2);
    }
};

}  // namespace

struct knn_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    knn_options opt{};

    std::shared_ptr<RefSet> ref;   // null until a reference set is given

    // workspace (grown on demand, or reserved up front with knn_reserve)
    unsigned char* ws = nullptr;
    size_t ws_bytes = 0;

    Counters* counters = nullptr;  // device
    int32_t* flag_host = nullptr;  // pinned host word: the error flag as a host-buffer search ends
    // host-buffer searches in parts: the side streams of parts after the
    // first, and the events that order them (start; each part's query
    // preparation done; each side part done)
    cudaStream_t pipe_stream[kMaxParts - 1] = {};
    cudaEvent_t pipe_start = nullptr, pipe_prep[kMaxParts - 1] = {}, pipe_done[kMaxParts - 1] = {};
    int64_t searches = 0;
    int64_t launches = 0;

    bool profiling = false;
    cudaEvent_t ev[kMaxStages + 1] = {};
    const char* stage_names[kMaxStages] = {};
    int nstages = 0;

    std::string last_error;

    // batches: captured graphs by batch signature, tuned launch configurations
    // by batch shape, the streams the captures fork over
    struct BatchGraph {
        cudaGraphExec_t exec = nullptr;
        int branches = 0;
        int sm_share = 0;
        int launches = 0;
        size_t nodes = 0;
        PersistBatch pb{};     // the persistent form: its descriptors (owned)
        bool persistent = false;
    };
    std::map<uint64_t, BatchGraph> graphs;
    std::map<uint64_t, std::pair<int, int>> tuned;   // shape -> (branches, sm_share)
    // persistent form: shape -> reference-split length per (d, k) bucket
    std::map<uint64_t, std::map<uint64_t, int64_t>> tuned_chunks;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t branch[16] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[16] = {}, t_ev[2] = {};
    knn_batch_info last_batch{};
    // per-stage time counters of the last persistent batch run (in the
    // workspace; cleared by the next search of any kind), and its stream
    unsigned long long* last_stage_ns = nullptr;
    cudaStream_t last_stage_stream = nullptr;

    // Mahalanobis distance: the Cholesky factor L of the inverse covariance
    // (device, float32, row-major), the whitened reference set built from
    // `ref` (rebuilt when `ref` or L changes) and a buffer for whitened queries
    int32_t mahal_d = 0;
    float* mahal_L = nullptr;
    std::shared_ptr<RefSet> mref;
    const RefSet* mref_src = nullptr;
    float* qw = nullptr;
    size_t qw_bytes = 0;
};

namespace {

knn_status cuda_fail(knn_ctx* h, cudaError_t err, const char* what) {
    if (h) {
        h->last_error = std::string(what) + ": " + cudaGetErrorString(err);
    }
    (void)cudaGetLastError();  // clear a sticky launch error if recoverable
    return (err == cudaErrorMemoryAllocation) ? KNN_ERR_OOM : KNN_ERR_CUDA;
}

#define KNN_CUDA(h, call)                                          \
    do {                                                           \
        cudaError_t err__ = (call);                                \
        if (err__ != cudaSuccess) return cuda_fail((h), err__, #call); \
    } while (0)

bool fault_inject_oom() {
    const char* v = std::getenv("KNN_FAULT_INJECT_OOM");
    return v && v[0] == '1';
}

void drop_graphs(knn_ctx* h) {
    for (auto& kv : h->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        persist_free(&kv.second.pb);
    }
    h->graphs.clear();
}

// Make sure the handle's workspace holds at least `bytes`.
knn_status ensure_workspace(knn_ctx* h, size_t bytes) {
    if (bytes <= h->ws_bytes) return KNN_OK;
    if (fault_inject_oom()) {
        h->last_error = "workspace allocation refused (KNN_FAULT_INJECT_OOM=1)";
        return KNN_ERR_OOM;
    }
    if (h->opt.workspace_limit > 0 && bytes > static_cast<size_t>(h->opt.workspace_limit)) {
        h->last_error = "workspace over the handle's limit";
        return KNN_ERR_OOM;
    }
    KNN_CUDA(h, cudaDeviceSynchronize());   // batch graphs may run on other streams
    drop_graphs(h);                          // they point into the old workspace
    if (h->ws) KNN_CUDA(h, cudaFree(h->ws));
    h->ws = nullptr;
    h->ws_bytes = 0;
    const size_t grow = bytes + bytes / 4;
    cudaError_t err = cudaMalloc(&h->ws, grow);
    if (err != cudaSuccess) {
        err = cudaMalloc(&h->ws, bytes);
        if (err != cudaSuccess) return cuda_fail(h, err, "cudaMalloc(workspace)");
        h->ws_bytes = bytes;
    } else {
        h->ws_bytes = grow;
    }
    return KNN_OK;
}

// Bump allocator over the workspace (256-byte aligned slices).
struct Carve {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t at = off;
        off += (bytes + 255) & ~static_cast<size_t>(255);
        return at;
    }
};

knn_status build_lowp_on(knn_ctx* h, std::shared_ptr<RefSet>& ref, int prec) {
    RefSet& rs = *ref;
    if (rs.lp_prec == prec && rs.R_lp) return KNN_OK;
    if (ref.use_count() > 1) {
        h->last_error = "the shared reference set holds another low-precision copy";
        return KNN_ERR_BUSY;
    }
    if (rs.R_lp) {
        KNN_CUDA(h, cudaFree(rs.R_lp));
        rs.R_lp = nullptr;
        rs.lp_prec = 0;
    }
    const int kp = tc_padded_dim(rs.d, prec);
    const size_t elt = (prec == kBF16) ? 2 : 4;
    KNN_CUDA(h, cudaMalloc(&rs.R_lp, static_cast<size_t>(rs.m) * kp * elt));
    int l = 0;
    KNN_CUDA(h, launch_prepare_ref(rs.R, rs.m, rs.d, kp, prec, rs.R_lp, rs.r_norms, rs.rmax2,
                                   h->stream, &l));
    h->launches += l;
    KNN_CUDA(h, cudaStreamSynchronize(h->stream));
    rs.kp = kp;
    rs.lp_prec = prec;
    return KNN_OK;
}

knn_status build_lowp(knn_ctx* h, int prec) { return build_lowp_on(h, h->ref, prec); }

// A reference set owning a float32 copy of R (m x d) and zeroed norm buffers;
// src_kind is the cudaMemcpy kind of the copy.
knn_status new_refset(knn_ctx* h, const float* R, int64_t m, int32_t d, cudaMemcpyKind src_kind,
                      std::shared_ptr<RefSet>* out) {
    auto rs = std::make_shared<RefSet>();
    rs->device = h->device;
    const size_t bytes = static_cast<size_t>(m) * d * sizeof(float);
    KNN_CUDA(h, cudaMalloc(&rs->R, bytes));
    // norms padded to whole 128-reference tiles (zero beyond m)
    const size_t mpad = static_cast<size_t>((m + 127) / 128 * 128);
    KNN_CUDA(h, cudaMalloc(&rs->r_norms, mpad * sizeof(float)));
    KNN_CUDA(h, cudaMalloc(&rs->rmax2, sizeof(uint32_t)));
    KNN_CUDA(h, cudaMemsetAsync(rs->r_norms, 0, mpad * sizeof(float), h->stream));
    KNN_CUDA(h, cudaMemsetAsync(rs->rmax2, 0, sizeof(uint32_t), h->stream));
    if (R) KNN_CUDA(h, cudaMemcpyAsync(rs->R, R, bytes, src_kind, h->stream));
    KNN_CUDA(h, cudaStreamSynchronize(h->stream));
    rs->m = m;
    rs->d = d;
    *out = std::move(rs);
    return KNN_OK;
}

// The whitened reference set of the Mahalanobis distance: R L, built from the
// current reference set when it or L changed since the last build.
knn_status ensure_mref(knn_ctx* h) {
    if (h->mref && h->mref_src == h->ref.get()) return KNN_OK;
    h->mref.reset();
    h->mref_src = nullptr;
    std::shared_ptr<RefSet> w;
    knn_status s = new_refset(h, nullptr, h->ref->m, h->ref->d, cudaMemcpyDeviceToDevice, &w);
    if (s != KNN_OK) return s;
    int l = 0;
    KNN_CUDA(h, launch_whiten(h->ref->R, h->ref->m, h->ref->d, h->mahal_L, w->R, h->stream, &l));
    KNN_CUDA(h, cudaStreamSynchronize(h->stream));
    h->launches += l;
    h->mref = std::move(w);
    h->mref_src = h->ref.get();
    return KNN_OK;
}

// True for page-locked host memory the GPU can address at the same pointer
// (cudaHostAlloc / cudaHostRegister under unified addressing).
bool host_mapped(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost && at.devicePointer == p;
}

// Cholesky factor of a symmetric positive definite d x d matrix (row-major,
// lower triangle read), in double: L[i][j] for j <= i, zero above.  Returns
// false when a pivot is not positive or a value is not finite.
bool cholesky_lower(const double* M, int32_t d, std::vector<double>* L) {
    L->assign(static_cast<size_t>(d) * d, 0.0);
    for (int32_t j = 0; j < d; ++j) {
        double s = M[static_cast<size_t>(j) * d + j];
        for (int32_t t = 0; t < j; ++t) s -= (*L)[static_cast<size_t>(j) * d + t] * (*L)[static_cast<size_t>(j) * d + t];
        if (!(s > 0.0) || !std::isfinite(s)) return false;
        const double ljj = std::sqrt(s);
        (*L)[static_cast<size_t>(j) * d + j] = ljj;
        for (int32_t i = j + 1; i < d; ++i) {
            double v = M[static_cast<size_t>(i) * d + j];
            for (int32_t t = 0; t < j; ++t) v -= (*L)[static_cast<size_t>(i) * d + t] * (*L)[static_cast<size_t>(j) * d + t];
            if (!std::isfinite(v)) return false;
            (*L)[static_cast<size_t>(i) * d + j] = v / ljj;
        }
    }
    return true;
}

int ceil_div(int64_t a, int64_t b) { return static_cast<int>((a + b - 1) / b); }

void stage(knn_ctx* h, cudaStream_t st, const char* name) {
    if (!h->profiling || h->nstages >= kMaxStages) return;
    h->stage_names[h->nstages] = name;
    cudaEventRecord(h->ev[h->nstages + 1], st);
    ++h->nstages;
}

// Everything a search of n queries decides before it launches: the form, the
// candidate count, the reference splits and the workspace layout.
struct SearchPlan {
    bool tensor = false;
    bool small = false;      // float32: all m distances per query in shared memory (knn_small.cu)
    int c_need = 0;          // small: the nearest keys a query must keep (c slots, c >= c_need)
    int prec = 0;
    int kp = 0;
    int c = 0;
    int S = 1;
    int64_t chunk = 0;
    TcPlan plan{};
    int64_t fb_grid = 1;
    size_t off_cand = 0, off_ql = 0, off_gmax = 0, off_lists = 0, off_counts = 0, off_qs = 0;
    size_t off_list = 0, off_scr = 0, off_fbdone = 0, off_q = 0, off_dist = 0, off_idx = 0;
    size_t bytes = 0;
};

// sm_share: how many SMs the search should fill on its own (all of them for a
// lone search; fewer when several run side by side in a batch).
knn_status plan_search_md(const knn_ctx* h, int64_t m, int32_t d, int precision, int64_t n, int32_t k,
                          knn_metric metric, int io_on_device, int sm_share, SearchPlan* sp,
                          int64_t fb_cap_bytes = 64LL << 20) {
    SearchPlan p;
    p.tensor = (metric == KNN_L2) && precision != KNN_FP32;
    p.prec = p.tensor ? (precision == KNN_BF16 ? kBF16 : kTF32) : 0;

    // candidates per query: k plus a margin (float32), rerank_factor * k (tensor cores)
    if (p.tensor) {
        p.c = h->opt.rerank_factor * k;
        if (p.c > (finalize_max_pool() - 32) / 2) p.c = (finalize_max_pool() - 32) / 2;
        if (p.c < k) return KNN_ERR_UNSUPPORTED;
    } else {
        const int margin = k / 4 > 8 ? k / 4 : 8;
        p.c = k + margin;
        if (p.c > cc_max_candidates()) p.c = cc_max_candidates();
        if (p.c > m) p.c = static_cast<int>(m);
        if (p.c < k) return KNN_ERR_UNSUPPORTED;
    }

    // float32 path: reference splits so that enough CTAs fill the GPU, each
    // split much larger than c, all splits' candidates within one finalize pool
    if (p.tensor) {
        p.kp = tc_padded_dim(d, p.prec);
        p.plan = tc_plan(n, m, d, p.kp, p.prec, p.c, sm_share);
        // rows too long for the tile, or a reference set too small for the
        // pilot (every reference would be appended to the lists): the float32
        // form, whose small-set select handles the latter faster and exactly.
        // Where both would run, the small-set select is kept while each SM's
        // share of its distance work (CTAs of eight queries, each over all m
        // references) stays small: its time grows with that share, the
        // tensor-core form's stays near 0.09 ms at these sizes (measured at
        // n = m = 2400: d = 32, 151k products per SM, 0.082 against 0.089 ms;
        // d = 64, 303k, 0.104 against 0.089 ms)
        const double small_share = static_cast<double>((n + 7) / 8) * static_cast<double>(m) *
                                   static_cast<double>(d) / static_cast<double>(sm_share);
        if (p.plan.stages == 0 ||
            (small_select_fits(m, d) && (!p.plan.pilot || small_share < kSmallSelectShare)))
            return plan_search_md(h, m, d, KNN_FP32, n, k, metric, io_on_device, sm_share, sp,
                                  fb_cap_bytes);
        p.S = p.plan.S;
        p.chunk = p.plan.chunk;
    } else if (small_select_fits(m, d)) {
        p.small = true;
        p.c_need = p.c;
        p.c = static_cast<int>(std::min<int64_t>(m, p.c + kSmallSelectSpare));
        p.S = 1;
        p.chunk = m;
    } else {
        int64_t chunk = 0;
        const int S = cc_plan_splits(n, m, p.c, sm_share, finalize_max_pool(), &chunk);
        if (static_cast<int64_t>(S) * p.c > finalize_max_pool()) return KNN_ERR_UNSUPPORTED;
        p.S = S;
        p.chunk = chunk;
    }

    // fallback grid: scratch of grid * m doubles, at most fb_cap_bytes
    p.fb_grid = fb_cap_bytes / (8 * m);
    if (p.fb_grid > 64) p.fb_grid = 64;
    if (p.fb_grid < 1) p.fb_grid = 1;

    // workspace layout
    Carve cv;
    if (p.tensor) {
        const size_t elt = (p.prec == kBF16) ? 2 : 4;
        p.off_ql = cv.take(static_cast<size_t>(n) * p.kp * elt);
        if (p.plan.pilot) p.off_gmax = cv.take(static_cast<size_t>(n) * p.plan.G * 4);
        p.off_lists = cv.take(static_cast<size_t>(n) * p.S * p.plan.groups * p.plan.cap *
                              sizeof(uint64_t));
        p.off_counts = cv.take(static_cast<size_t>(n) * p.S * p.plan.groups * sizeof(int32_t));
        p.off_qs = cv.take(static_cast<size_t>(n) * sizeof(float));
    } else {
        p.off_cand = cv.take(static_cast<size_t>(n) * p.S * p.c * sizeof(uint64_t));
    }
    p.off_list = cv.take(static_cast<size_t>(n) * sizeof(int32_t));
    p.off_scr = cv.take(static_cast<size_t>(p.fb_grid) * m * sizeof(double));
    p.off_fbdone = cv.take(static_cast<size_t>(p.fb_grid) * sizeof(int32_t));
    if (!io_on_device) {
        p.off_q = cv.take(static_cast<size_t>(n) * d * sizeof(float));
        p.off_dist = cv.take(static_cast<size_t>(n) * k * sizeof(float));
        p.off_idx = cv.take(static_cast<size_t>(n) * k * sizeof(int32_t));
    }
    p.bytes = cv.off;
    *sp = p;
    return KNN_OK;
}

knn_status plan_search(const knn_ctx* h, int64_t n, int32_t k, knn_metric metric, int io_on_device,
                       SearchPlan* sp) {
    return plan_search_md(h, h->ref->m, h->ref->d, h->opt.precision, n, k, metric, io_on_device,
                          h->num_sms, sp);
}

// The reference data one search reads: a handle's reference set, or the
// arrays of a batch instance (prepared inside the batch's own workspace).
struct RefView {
    const float* R;
    int64_t m;
    int32_t d;
    void* R_lp;
    int32_t kp;
    const uint32_t* rmax2;
};

// Enqueue the kernels of one planned search on st: Q, dd, id on the device,
// ws the search's workspace, fallback_count a device int of its own.
// Qd: the queries as the kernels read them.  Q_copy (tensor-core plans only):
// when given, Qd is host memory read once by the query preparation, which
// leaves a float32 device copy there for the later stages.
knn_status enqueue_search(knn_ctx* h, const SearchPlan& sp, const RefView& rv, const float* Qd,
                          int64_t n, int32_t k, knn_metric metric, float* dd, int32_t* id,
                          unsigned char* ws, int32_t* fallback_count, cudaStream_t st, int* l,
                          bool stages, float* Q_copy = nullptr, cudaEvent_t prep_done = nullptr) {
    const int64_t m = rv.m;
    const int32_t d = rv.d;
    const int S = sp.S, c = sp.c;
    Counters* ctr = h->counters;
    auto mark = [&](const char* name) {
        if (stages) stage(h, st, name);
    };
    KNN_CUDA(h, cudaMemsetAsync(fallback_count, 0, sizeof(int32_t), st));
    FinalizeArgs fa{};
    if (sp.tensor) {
        const TcPlan& plan = sp.plan;
        const int prec = sp.prec;
        void* Ql = ws + sp.off_ql;
        uint64_t* lists = reinterpret_cast<uint64_t*>(ws + sp.off_lists);
        int32_t* counts = reinterpret_cast<int32_t*>(ws + sp.off_counts);
        HitScale qs;
        qs.rmax2 = rv.rmax2;
        qs.qscale = reinterpret_cast<float*>(ws + sp.off_qs);
        HitScale qs_prep = qs;   // the threshold pass sets B when there is one
        if (plan.pilot) qs_prep.qscale = nullptr;
        KNN_CUDA(h, launch_prepare_query(Qd, n, d, rv.kp, prec, Ql, qs_prep, Q_copy, st, l));
        if (Q_copy) Qd = Q_copy;
        mark("prepare_q");
        if (prep_done) KNN_CUDA(h, cudaEventRecord(prep_done, st));
        if (plan.pilot) {
            uint32_t* gmax = reinterpret_cast<uint32_t*>(ws + sp.off_gmax);
            KNN_CUDA(h, launch_tc_pilot(plan, Ql, n, rv.R_lp, m, rv.kp, prec, gmax, &ctr->error_flag,
                                        st, l));
            mark("tc_pilot");
            KNN_CUDA(h, launch_tc_threshold(plan, gmax, n, d, rv.kp, prec, Ql, qs, st, l));
            mark("tc_threshold");
        }
        KNN_CUDA(h, launch_tc_filter(plan, Ql, n, rv.R_lp, m, rv.kp, prec, lists, counts, qs.qscale,
                                     &ctr->error_flag, st, l));
        mark("tc_filter");
        fa.use_hits = 1;
        fa.hits.keys = lists;
        fa.hits.counts = counts;
        fa.hits.S = plan.groups * S;   // one list per (split, epilogue column group)
        fa.hits.cap = plan.cap;
        fa.hits.c = c;
        fa.cand.exact = 0;
        fa.cand.S = 1;
        fa.cand.c = c;
    } else {
        CandidateSet cs;
        cs.keys = reinterpret_cast<uint64_t*>(ws + sp.off_cand);
        cs.n = n;
        cs.S = S;
        cs.c = c;
        cs.chunk = sp.chunk;
        cs.exact = 1;
        if (sp.small) {
            KNN_CUDA(h, launch_small_select(Qd, n, rv.R, m, d, metric, sp.c_need, cs, st, l));
            mark("small_select");
        } else {
            KNN_CUDA(h, launch_cc_select(Qd, n, rv.R, m, d, metric, cs, st, l));
            mark("cc_select");
        }
        fa.use_hits = 0;
        fa.cand = cs;
    }
    fa.Q = Qd;
    fa.R = rv.R;
    fa.n = n;
    fa.m = m;
    fa.d = d;
    fa.k = k;
    fa.metric = metric;
    fa.dist_out = dd;
    fa.idx_out = id;
    fa.fallback_count = fallback_count;
    fa.fallback_list = reinterpret_cast<int32_t*>(ws + sp.off_list);
    fa.recheck_counter = &ctr->recheck_total;
    fa.fallback_total = &ctr->fallback_total;
    fa.fallback_reason = ctr->fallback_reason;
    fa.fb_done = reinterpret_cast<int32_t*>(ws + sp.off_fbdone);
    fa.fb_slots = static_cast<int32_t>(sp.fb_grid);
    KNN_CUDA(h, launch_finalize(fa, st, l));
    mark("finalize");
    KNN_CUDA(h, launch_fallback(fa, reinterpret_cast<double*>(ws + sp.off_scr),
                                static_cast<int32_t>(sp.fb_grid), fa.fb_done, st, l));
    mark("fallback");
    return KNN_OK;
}

knn_status check_search_args(const knn_ctx* h, int64_t n, int32_t d, int32_t k, knn_metric metric) {
    if (!h) return KNN_ERR_INVALID;
    if (n < 0 || k < 1 ||
        (metric != KNN_L2 && metric != KNN_L1 && metric != KNN_LINF && metric != KNN_MAHALANOBIS))
        return KNN_ERR_INVALID;
    if (!h->ref) return KNN_ERR_NOREF;
    if (d != h->ref->d || k > h->ref->m) return KNN_ERR_INVALID;
    if (metric == KNN_MAHALANOBIS && h->mahal_d != d) return KNN_ERR_INVALID;
    if (k > KNN_K_MAX) return KNN_ERR_UNSUPPORTED;
    if (n > 0x7fffffffLL) return KNN_ERR_UNSUPPORTED;
    return KNN_OK;
}

bool valid_options(const knn_options& o) {
    return !(o.precision < KNN_FP32 || o.precision > KNN_BF16 || o.rerank_factor < 1 ||
             o.rerank_factor > 64 || o.workspace_limit < 0);
}


// ------------------------------------------------------------------ batches

uint64_t mix64(uint64_t h, uint64_t v) {
    return h ^ (v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2));
}

// Shape signature (and, with pointers, the exact batch) of a batch.
uint64_t batch_signature(const knn_ctx* h, const knn_instance* inst, int32_t count, bool pointers) {
    uint64_t g = mix64(0x51ed270b27e3c9e5ull, static_cast<uint64_t>(count));
    g = mix64(g, static_cast<uint64_t>(h->opt.precision) * 131 + h->opt.rerank_factor);
    for (int32_t i = 0; i < count; ++i) {
        const knn_instance& x = inst[i];
        g = mix64(g, static_cast<uint64_t>(x.m));
        g = mix64(g, static_cast<uint64_t>(x.n));
        g = mix64(g, (static_cast<uint64_t>(x.d) << 32) | static_cast<uint32_t>(x.k));
        g = mix64(g, static_cast<uint64_t>(x.metric));
        if (pointers) {
            g = mix64(g, reinterpret_cast<uintptr_t>(x.R));
            g = mix64(g, reinterpret_cast<uintptr_t>(x.Q));
            g = mix64(g, reinterpret_cast<uintptr_t>(x.dist_out));
            g = mix64(g, reinterpret_cast<uintptr_t>(x.idx_out));
        }
    }
    return g;
}

knn_status check_instance(const knn_instance& x) {
    if (x.n < 0 || x.m < 1 || x.d < 1 || x.k < 1 || x.k > x.m ||
        (x.metric != KNN_L2 && x.metric != KNN_L1 && x.metric != KNN_LINF))
        return KNN_ERR_INVALID;
    if (!x.R || (x.n > 0 && (!x.Q || !x.dist_out || !x.idx_out))) return KNN_ERR_INVALID;
    if (x.k > KNN_K_MAX || x.m > 0x7fffffffLL || x.n > 0x7fffffffLL) return KNN_ERR_UNSUPPORTED;
    return KNN_OK;
}

// Plans and workspace slices of every instance of a batch.
struct BatchPlan {
    std::vector<SearchPlan> sp;
    std::vector<size_t> base, fbc, lp, rmax;
    size_t bytes = 0;
};

knn_status plan_batch(const knn_ctx* h, const knn_instance* inst, int32_t count, int sm_share,
                      BatchPlan* bp) {
    Carve cv;
    bp->sp.resize(count);
    bp->base.assign(count, 0);
    bp->fbc.assign(count, 0);
    bp->lp.assign(count, 0);
    bp->rmax.assign(count, 0);
    for (int32_t i = 0; i < count; ++i) {
        const knn_instance& x = inst[i];
        if (x.n == 0) continue;
        SearchPlan& sp = bp->sp[i];
        knn_status s = plan_search_md(h, x.m, x.d, h->opt.precision, x.n, x.k,
                                      static_cast<knn_metric>(x.metric), 1, sm_share, &sp,
                                      4LL << 20);
        if (s != KNN_OK) return s;
        bp->base[i] = cv.take(sp.bytes);
        bp->fbc[i] = cv.take(sizeof(int32_t));
        if (sp.tensor) {
            const size_t elt = (sp.prec == kBF16) ? 2 : 4;
            bp->lp[i] = cv.take(static_cast<size_t>(x.m) * sp.kp * elt);
            bp->rmax[i] = cv.take(sizeof(uint32_t));
        }
    }
    bp->bytes = cv.off;
    return KNN_OK;
}

// Enqueue instance i of a planned batch on st (its low-precision reference
// copy first, for the tensor-core forms).
knn_status enqueue_instance(knn_ctx* h, const knn_instance& x, const BatchPlan& bp, int32_t i,
                            cudaStream_t st, int* l) {
    if (x.n == 0) return KNN_OK;
    const SearchPlan& sp = bp.sp[i];
    unsigned char* ws = h->ws;
    RefView rv{x.R, x.m, x.d, nullptr, 0, nullptr};
    if (sp.tensor) {
        rv.R_lp = ws + bp.lp[i];
        rv.kp = sp.kp;
        rv.rmax2 = reinterpret_cast<uint32_t*>(ws + bp.rmax[i]);
        KNN_CUDA(h, launch_prepare_ref(x.R, x.m, x.d, sp.kp, sp.prec, rv.R_lp, nullptr,
                                       reinterpret_cast<uint32_t*>(ws + bp.rmax[i]), st, l));
    }
    return enqueue_search(h, sp, rv, x.Q, x.n, x.k, static_cast<knn_metric>(x.metric), x.dist_out,
                          x.idx_out, ws + bp.base[i], reinterpret_cast<int32_t*>(ws + bp.fbc[i]),
                          st, l, false);
}

// The side streams and events of a host-buffer search run in parts.
knn_status pipe_streams(knn_ctx* h) {
    if (h->pipe_start) return KNN_OK;
    for (int i = 0; i < kMaxParts - 1; ++i) {
        KNN_CUDA(h, cudaStreamCreateWithFlags(&h->pipe_stream[i], cudaStreamNonBlocking));
        KNN_CUDA(h, cudaEventCreateWithFlags(&h->pipe_prep[i], cudaEventDisableTiming));
        KNN_CUDA(h, cudaEventCreateWithFlags(&h->pipe_done[i], cudaEventDisableTiming));
    }
    KNN_CUDA(h, cudaEventCreateWithFlags(&h->pipe_start, cudaEventDisableTiming));
    return KNN_OK;
}

knn_status batch_streams(knn_ctx* h) {
    if (h->cap_stream) return KNN_OK;
    KNN_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    for (int b = 0; b < 16; ++b) {
        KNN_CUDA(h, cudaStreamCreateWithFlags(&h->branch[b], cudaStreamNonBlocking));
        KNN_CUDA(h, cudaEventCreateWithFlags(&h->join_ev[b], cudaEventDisableTiming));
    }
    KNN_CUDA(h, cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
    KNN_CUDA(h, cudaEventCreate(&h->t_ev[0]));
    KNN_CUDA(h, cudaEventCreate(&h->t_ev[1]));
    return KNN_OK;
}

// Capture the batch into one graph: the instances spread over `branches`
// parallel branches, largest work first onto the least loaded branch.
knn_status capture_batch(knn_ctx* h, const knn_instance* inst, int32_t count, const BatchPlan& bp,
                         int branches, knn_ctx::BatchGraph* out) {
    knn_status s = batch_streams(h);
    if (s != KNN_OK) return s;
    if (branches < 1) branches = 1;
    if (branches > 16) branches = 16;
    std::vector<int32_t> order(count);
    for (int32_t i = 0; i < count; ++i) order[i] = i;
    auto work = [&](int32_t i) {
        return static_cast<double>(inst[i].n) * inst[i].m * inst[i].d + 1e6;
    };
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return work(a) > work(b); });
    std::vector<double> load(branches, 0.0);
    KNN_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed));
    cudaError_t err = cudaEventRecord(h->fork_ev, h->cap_stream);
    for (int b = 0; err == cudaSuccess && b < branches; ++b)
        err = cudaStreamWaitEvent(h->branch[b], h->fork_ev, 0);
    int l = 0;
    s = (err == cudaSuccess) ? KNN_OK : cuda_fail(h, err, "batch fork");
    for (int32_t t = 0; s == KNN_OK && t < count; ++t) {
        const int32_t i = order[t];
        const int b = static_cast<int>(std::min_element(load.begin(), load.end()) - load.begin());
        load[b] += work(i);
        s = enqueue_instance(h, inst[i], bp, i, h->branch[b], &l);
    }
    // join every branch even after an error, so that the capture can end
    for (int b = 0; b < branches; ++b) {
        cudaEventRecord(h->join_ev[b], h->branch[b]);
        cudaStreamWaitEvent(h->cap_stream, h->join_ev[b], 0);
    }
    cudaGraph_t graph = nullptr;
    err = cudaStreamEndCapture(h->cap_stream, &graph);
    if (s != KNN_OK || err != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        (void)cudaGetLastError();
        return s != KNN_OK ? s : cuda_fail(h, err, "cudaStreamEndCapture");
    }
    size_t nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &nodes);
    cudaGraphExec_t exec = nullptr;
    err = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) return cuda_fail(h, err, "cudaGraphInstantiate");
    out->exec = exec;
    out->branches = branches;
    out->launches = l;
    out->nodes = nodes;
    return KNN_OK;
}

// Plan, size the workspace and capture one configuration.
knn_status build_batch(knn_ctx* h, const knn_instance* inst, int32_t count, int branches,
                       int sm_share, knn_ctx::BatchGraph* out) {
    BatchPlan bp;
    knn_status s = plan_batch(h, inst, count, sm_share, &bp);
    if (s != KNN_OK) return s;
    s = ensure_workspace(h, bp.bytes);
    if (s != KNN_OK) return s;
    s = capture_batch(h, inst, count, bp, branches, out);
    if (s == KNN_OK) out->sm_share = sm_share;
    return s;
}

// ------------------------------------------------------- persistent batches

// Bound of every wait of the persistent kernel in a normal run.
constexpr uint64_t kPersistWaitNs = 1000000000ull;

// (d, k) bucket of an instance: the unit the autotuner picks split lengths for.
uint64_t bucket_of(const knn_instance& x) {
    return (static_cast<uint64_t>(static_cast<uint32_t>(x.d)) << 32) | static_cast<uint32_t>(x.k);
}

// True when every instance can take the persistent tensor-core form.
bool persistent_eligible(const knn_ctx* h, const knn_instance* inst, int32_t count) {
    if (h->opt.precision == KNN_FP32) return false;
    for (int32_t i = 0; i < count; ++i)
        if (inst[i].metric != KNN_L2) return false;
    return true;
}

std::vector<PersistInst> persist_inputs(const knn_instance* inst, int32_t count,
                                        const std::map<uint64_t, int64_t>& chunks) {
    std::vector<PersistInst> v(count);
    for (int32_t i = 0; i < count; ++i) {
        const knn_instance& x = inst[i];
        auto it = chunks.find(bucket_of(x));
        v[i] = PersistInst{x.R, x.m, x.Q, x.n, x.d, x.k, x.dist_out, x.idx_out,
                           it == chunks.end() ? 0 : it->second};
    }
    return v;
}

// Plan, size the workspace, build and capture (counters reset, ready word
// set, one kernel) one persistent batch.  KNN_ERR_UNSUPPORTED when some
// instance cannot run in that form.
knn_status build_persistent(knn_ctx* h, const std::vector<PersistInst>& pin, knn_ctx::BatchGraph* out) {
    const int prec = h->opt.precision == KNN_BF16 ? kBF16 : kTF32;
    PersistPlan pp;
    cudaError_t err = persist_plan(pin, prec, h->opt.rerank_factor, h->num_sms, &pp);
    if (err == cudaErrorNotSupported) return KNN_ERR_UNSUPPORTED;
    if (err != cudaSuccess) return cuda_fail(h, err, "persist_plan");
    knn_status s = ensure_workspace(h, pp.ws_bytes);
    if (s != KNN_OK) return s;
    s = batch_streams(h);
    if (s != KNN_OK) return s;
    PersistCounters ctr{&h->counters->error_flag, &h->counters->recheck_total,
                        &h->counters->fallback_total, h->counters->fallback_reason};
    PersistBatch pb;
    KNN_CUDA(h, persist_build(pin, pp, prec, h->ws, ctr, &pb));
    KNN_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed));
    err = persist_launch(pb, h->num_sms, true, kPersistWaitNs, h->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t err2 = cudaStreamEndCapture(h->cap_stream, &graph);
    if (err != cudaSuccess || err2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        persist_free(&pb);
        (void)cudaGetLastError();
        return cuda_fail(h, err != cudaSuccess ? err : err2, "persistent batch capture");
    }
    size_t nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &nodes);
    cudaGraphExec_t exec = nullptr;
    err = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) {
        persist_free(&pb);
        return cuda_fail(h, err, "cudaGraphInstantiate");
    }
    out->exec = exec;
    out->pb = pb;
    out->persistent = true;
    out->branches = 1;
    out->sm_share = h->num_sms;
    out->launches = 1;
    out->nodes = nodes;
    return KNN_OK;
}

// Split lengths the autotuner tries for every (d, k) bucket (0: the planner's
// own choice, by how full the last wave of a lone search would be).
constexpr int64_t kChunkChoices[] = {0, 16384, 32768, 65536};

// Time each split length on the sub-batch of each (d, k) bucket and keep the
// fastest per bucket.
knn_status tune_persistent(knn_ctx* h, const knn_instance* inst, int32_t count, cudaStream_t st,
                           std::map<uint64_t, int64_t>* best, float* tune_ms) {
    std::map<uint64_t, std::vector<knn_instance>> buckets;
    for (int32_t i = 0; i < count; ++i)
        if (inst[i].n > 0) buckets[bucket_of(inst[i])].push_back(inst[i]);
    for (auto& kv : buckets) {
        float best_ms = 0.f;
        int64_t best_chunk = 0;
        bool have = false;
        for (int64_t ch : kChunkChoices) {
            std::map<uint64_t, int64_t> one{{kv.first, ch}};
            std::vector<PersistInst> pin =
                persist_inputs(kv.second.data(), static_cast<int32_t>(kv.second.size()), one);
            knn_ctx::BatchGraph g;
            knn_status s = build_persistent(h, pin, &g);
            if (s != KNN_OK) return s;
            KNN_CUDA(h, cudaGraphLaunch(g.exec, st));   // warm
            KNN_CUDA(h, cudaEventRecord(h->t_ev[0], st));
            KNN_CUDA(h, cudaGraphLaunch(g.exec, st));
            KNN_CUDA(h, cudaEventRecord(h->t_ev[1], st));
            KNN_CUDA(h, cudaEventSynchronize(h->t_ev[1]));
            float ms = 0.f;
            KNN_CUDA(h, cudaEventElapsedTime(&ms, h->t_ev[0], h->t_ev[1]));
            *tune_ms += 2.f * ms;
            cudaGraphExecDestroy(g.exec);
            persist_free(&g.pb);
            if (!have || ms < best_ms) {
                best_ms = ms;
                best_chunk = ch;
                have = true;
            }
        }
        (*best)[kv.first] = best_chunk;
    }
    return KNN_OK;
}

}  // namespace

extern "C" {

void knn_options_default(knn_options* opt) {
    if (!opt) return;
    opt->precision = KNN_FP32;
    opt->rerank_factor = 4;
    opt->workspace_limit = 0;
}

static knn_status new_handle(knn_handle* out, int device, const knn_options& o) {
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        (void)cudaGetLastError();
        return KNN_ERR_CUDA;
    }
    knn_ctx* h = new (std::nothrow) knn_ctx();
    if (!h) return KNN_ERR_OOM;
    h->device = device;
    h->opt = o;
    cudaError_t err = cudaSetDevice(device);
    if (err == cudaSuccess)
        err = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaMalloc(&h->counters, sizeof(Counters));
    if (err == cudaSuccess) err = cudaMemset(h->counters, 0, sizeof(Counters));
    if (err == cudaSuccess) err = cudaHostAlloc(&h->flag_host, sizeof(int32_t), cudaHostAllocDefault);
    for (int i = 0; err == cudaSuccess && i <= kMaxStages; ++i) err = cudaEventCreate(&h->ev[i]);
    if (err != cudaSuccess) {
        knn_destroy(h);
        (void)cudaGetLastError();
        return err == cudaErrorMemoryAllocation ? KNN_ERR_OOM : KNN_ERR_CUDA;
    }
    *out = h;
    return KNN_OK;
}

knn_status knn_create(knn_handle* out, int device, const knn_options* opt) {
    if (!out) return KNN_ERR_INVALID;
    *out = nullptr;
    knn_options o;
    knn_options_default(&o);
    if (opt) o = *opt;
    if (!valid_options(o)) return KNN_ERR_INVALID;
    return new_handle(out, device, o);
}

knn_status knn_create_shared(knn_handle* out, knn_handle src, const knn_options* opt) {
    if (!out) return KNN_ERR_INVALID;
    *out = nullptr;
    if (!src) return KNN_ERR_INVALID;
    knn_options o = src->opt;
    if (opt) {
        if (opt->precision != src->opt.precision) return KNN_ERR_INVALID;
        o = *opt;
    }
    if (!valid_options(o)) return KNN_ERR_INVALID;
    knn_status s = new_handle(out, src->device, o);
    if (s != KNN_OK) return s;
    (*out)->ref = src->ref;
    return KNN_OK;
}

knn_status knn_destroy(knn_handle h) {
    if (!h) return KNN_OK;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    h->ref.reset();
    if (h->cap_stream) cudaStreamSynchronize(h->cap_stream);
    for (int b = 0; b < 16; ++b) if (h->branch[b]) cudaStreamSynchronize(h->branch[b]);
    drop_graphs(h);
    for (int b = 0; b < 16; ++b) {
        if (h->branch[b]) cudaStreamDestroy(h->branch[b]);
        if (h->join_ev[b]) cudaEventDestroy(h->join_ev[b]);
    }
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (int i = 0; i < kMaxParts - 1; ++i) {
        if (h->pipe_stream[i]) {
            cudaStreamSynchronize(h->pipe_stream[i]);
            cudaStreamDestroy(h->pipe_stream[i]);
        }
        if (h->pipe_prep[i]) cudaEventDestroy(h->pipe_prep[i]);
        if (h->pipe_done[i]) cudaEventDestroy(h->pipe_done[i]);
    }
    if (h->pipe_start) cudaEventDestroy(h->pipe_start);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->t_ev[0]) cudaEventDestroy(h->t_ev[0]);
    if (h->t_ev[1]) cudaEventDestroy(h->t_ev[1]);
    if (h->ws) cudaFree(h->ws);
    if (h->counters) cudaFree(h->counters);
    if (h->flag_host) cudaFreeHost(h->flag_host);
    h->mref.reset();
    if (h->mahal_L) cudaFree(h->mahal_L);
    if (h->qw) cudaFree(h->qw);
    for (int i = 0; i <= kMaxStages; ++i)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return KNN_OK;
}

knn_status knn_set_reference(knn_handle h, const float* R, int64_t m, int32_t d, int r_on_device) {
    if (!h || !R || m < 1 || d < 1 || m > 0x7fffffffLL) return KNN_ERR_INVALID;
    KNN_CUDA(h, cudaSetDevice(h->device));
    KNN_CUDA(h, cudaStreamSynchronize(h->stream));
    h->ref.reset();   // a shared set stays with the other handles
    h->mref.reset();
    h->mref_src = nullptr;
    std::shared_ptr<RefSet> rs;
    knn_status s0 = new_refset(h, R, m, d,
                               r_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, &rs);
    if (s0 != KNN_OK) return s0;
    h->ref = std::move(rs);   // the handle is the set's only owner until it is shared
    if (h->opt.precision != KNN_FP32) {
        knn_status s = build_lowp(h, h->opt.precision == KNN_BF16 ? kBF16 : kTF32);
        if (s != KNN_OK) {
            h->ref.reset();
            return s;
        }
    }
    return KNN_OK;
}

knn_status knn_set_mahalanobis(knn_handle h, const double* S_inv, int32_t d) {
    if (!h) return KNN_ERR_INVALID;
    KNN_CUDA(h, cudaSetDevice(h->device));
    KNN_CUDA(h, cudaStreamSynchronize(h->stream));
    h->mref.reset();
    h->mref_src = nullptr;
    if (!S_inv) {
        if (h->mahal_L) KNN_CUDA(h, cudaFree(h->mahal_L));
        h->mahal_L = nullptr;
        h->mahal_d = 0;
        return KNN_OK;
    }
    if (d < 1) return KNN_ERR_INVALID;
    if (whiten_smem_bytes(d) > 227 * 1024) {
        h->last_error = "Mahalanobis distance: dimension above what the whitening kernel stages";
        return KNN_ERR_UNSUPPORTED;
    }
    std::vector<double> L;
    if (!cholesky_lower(S_inv, d, &L)) {
        h->last_error = "Mahalanobis matrix is not symmetric positive definite (Cholesky pivot <= 0)";
        return KNN_ERR_INVALID;
    }
    std::vector<float> Lf(L.size());
    for (size_t i = 0; i < L.size(); ++i) Lf[i] = static_cast<float>(L[i]);
    if (h->mahal_L && h->mahal_d != d) {
        KNN_CUDA(h, cudaFree(h->mahal_L));
        h->mahal_L = nullptr;
    }
    if (!h->mahal_L) KNN_CUDA(h, cudaMalloc(&h->mahal_L, Lf.size() * sizeof(float)));
    KNN_CUDA(h, cudaMemcpy(h->mahal_L, Lf.data(), Lf.size() * sizeof(float), cudaMemcpyHostToDevice));
    h->mahal_d = d;
    return KNN_OK;
}

knn_status knn_set_precision(knn_handle h, int32_t precision) {
    if (!h || precision < KNN_FP32 || precision > KNN_BF16) return KNN_ERR_INVALID;
    KNN_CUDA(h, cudaSetDevice(h->device));
    if (precision != KNN_FP32 && h->ref) {
        const int prec = precision == KNN_BF16 ? kBF16 : kTF32;
        knn_status s = build_lowp(h, prec);
        if (s != KNN_OK) return s;
    }
    h->opt.precision = precision;
    return KNN_OK;
}

knn_status knn_workspace_size(knn_handle h, int64_t n, int32_t d, int32_t k, knn_metric metric,
                              int io_on_device, int64_t* bytes) {
    if (!bytes) return KNN_ERR_INVALID;
    knn_status s = check_search_args(h, n, d, k, metric);
    if (s != KNN_OK) return s;
    if (n == 0) {
        *bytes = 0;
        return KNN_OK;
    }
    SearchPlan sp;
    // a Mahalanobis search is a Euclidean search of whitened points
    s = plan_search(h, n, k, metric == KNN_MAHALANOBIS ? KNN_L2 : metric, io_on_device, &sp);
    if (s != KNN_OK) return s;
    *bytes = static_cast<int64_t>(sp.bytes);
    return KNN_OK;
}

knn_status knn_reserve(knn_handle h, int64_t bytes) {
    if (!h || bytes < 0) return KNN_ERR_INVALID;
    KNN_CUDA(h, cudaSetDevice(h->device));
    return ensure_workspace(h, static_cast<size_t>(bytes));
}

knn_status knn_search(knn_handle h, const float* Q, int64_t n, int32_t d, int32_t k,
                      knn_metric metric, float* dist_out, int32_t* idx_out, int io_on_device,
                      void* cuda_stream) {
    knn_status s0 = check_search_args(h, n, d, k, metric);
    if (s0 != KNN_OK) return s0;
    h->last_stage_ns = nullptr;
    if (n > 0 && (!Q || !dist_out || !idx_out)) return KNN_ERR_INVALID;
    if (n == 0) return KNN_OK;
    KNN_CUDA(h, cudaSetDevice(h->device));
    cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : h->stream;
    // Mahalanobis: a Euclidean search of whitened queries against the
    // whitened reference set
    const bool mahal = metric == KNN_MAHALANOBIS;
    if (mahal) {
        knn_status sm = ensure_mref(h);
        if (sm != KNN_OK) return sm;
        metric = KNN_L2;
    }
    std::shared_ptr<RefSet>& refp = mahal ? h->mref : h->ref;
    RefSet& rs = *refp;
    const int64_t m = rs.m;

    SearchPlan sp;
    knn_status s = plan_search(h, n, k, metric, io_on_device, &sp);
    if (s != KNN_OK) return s;
    if (sp.tensor) {
        s = build_lowp_on(h, refp, sp.prec);
        if (s != KNN_OK) return s;
    }
    if (mahal && h->qw_bytes < static_cast<size_t>(n) * d * sizeof(float)) {
        KNN_CUDA(h, cudaStreamSynchronize(st));
        if (h->qw) KNN_CUDA(h, cudaFree(h->qw));
        h->qw = nullptr;
        h->qw_bytes = 0;
        KNN_CUDA(h, cudaMalloc(&h->qw, static_cast<size_t>(n) * d * sizeof(float)));
        h->qw_bytes = static_cast<size_t>(n) * d * sizeof(float);
    }
    s = ensure_workspace(h, sp.bytes);
    if (s != KNN_OK) return s;
    unsigned char* ws = h->ws;

    const float* Qd = Q;
    float* dd = dist_out;
    int32_t* id = idx_out;
    h->nstages = 0;
    if (h->profiling) cudaEventRecord(h->ev[0], st);
    // Host buffers.  Pinned ones are read and written by the kernels directly
    // over the CPU-GPU link (the tensor-core query preparation reads Q once and
    // keeps a device copy; the finalize writes the outputs in place); pageable
    // ones (and Q of a float32 or Mahalanobis search) go through copies.
    float* q_copy = nullptr;
    bool out_direct = false;
    if (!io_on_device) {
        const bool q_direct = !mahal && sp.tensor && host_mapped(Q);
        out_direct = host_mapped(dist_out) && host_mapped(idx_out);
        if (q_direct) {
            q_copy = reinterpret_cast<float*>(ws + sp.off_q);
        } else {
            Qd = reinterpret_cast<float*>(ws + sp.off_q);
            KNN_CUDA(h, cudaMemcpyAsync(const_cast<float*>(Qd), Q, static_cast<size_t>(n) * d * 4,
                                        cudaMemcpyHostToDevice, st));
            stage(h, st, "h2d");
        }
        if (!out_direct) {
            dd = reinterpret_cast<float*>(ws + sp.off_dist);
            id = reinterpret_cast<int32_t*>(ws + sp.off_idx);
        }
    }

    Counters* ctr = h->counters;
    int l = 0;
    if (mahal) {
        KNN_CUDA(h, launch_whiten(Qd, n, d, h->mahal_L, h->qw, st, &l));
        Qd = h->qw;
        stage(h, st, "whiten_q");
    }
    RefView rv{rs.R, rs.m, rs.d, rs.R_lp, rs.kp, rs.rmax2};
    // Queries and outputs both in pinned host memory, read and written in
    // place: the link moves the queries at a fraction of the rate the kernels
    // use them, so a large search runs in parts (whole 128-query tiles), each
    // on its own stream, each part's query preparation starting when the one
    // before it ends.  The link then carries a part's queries while the parts
    // before it compute.  Only when the parts' workspaces fit the one this
    // search already has, and no stage profiling is on.
    int parts = 1;
    SearchPlan pp[kMaxParts];
    size_t poff[kMaxParts] = {};
    int64_t pb[kMaxParts + 1] = {};
    if (q_copy && out_direct && !h->profiling) {
        for (int np = static_cast<int>(std::min<int64_t>(kMaxParts, n / kPartMinQueries)); np > 1;
             np = np > 2 ? 2 : 1) {
            bool ok = true;
            size_t total = 0;
            for (int j = 0; j <= np; ++j) pb[j] = j == np ? n : (n * j / np + 127) / 128 * 128;
            for (int j = 0; j < np && ok; ++j) {
                ok = plan_search(h, pb[j + 1] - pb[j], k, metric, 0, &pp[j]) == KNN_OK && pp[j].tensor;
                poff[j] = total;
                total += (pp[j].bytes + 255) / 256 * 256;
            }
            if (ok && total <= h->ws_bytes) {
                parts = np;
                break;
            }
        }
    }
    if (parts > 1) {
        s = pipe_streams(h);
        if (s != KNN_OK) return s;
        KNN_CUDA(h, cudaEventRecord(h->pipe_start, st));
        for (int j = 0; j < parts; ++j) {
            cudaStream_t sj = j == 0 ? st : h->pipe_stream[j - 1];
            if (j > 0) {
                KNN_CUDA(h, cudaStreamWaitEvent(sj, h->pipe_start, 0));
                KNN_CUDA(h, cudaStreamWaitEvent(sj, h->pipe_prep[j - 1], 0));
            }
            unsigned char* wj = ws + poff[j];
            int32_t* fc = j == 0 ? &ctr->fallback_count : &ctr->fallback_part[j - 1];
            s = enqueue_search(h, pp[j], rv, Q + pb[j] * d, pb[j + 1] - pb[j], k, metric,
                               dist_out + pb[j] * k, idx_out + pb[j] * k, wj, fc, sj, &l, false,
                               reinterpret_cast<float*>(wj + pp[j].off_q),
                               j + 1 < parts ? h->pipe_prep[j] : nullptr);
            if (s != KNN_OK) return s;
        }
        for (int j = 1; j < parts; ++j) {
            KNN_CUDA(h, cudaEventRecord(h->pipe_done[j - 1], h->pipe_stream[j - 1]));
            KNN_CUDA(h, cudaStreamWaitEvent(st, h->pipe_done[j - 1], 0));
        }
    } else {
        s = enqueue_search(h, sp, rv, Qd, n, k, metric, dd, id, ws, &ctr->fallback_count, st, &l,
                           true, q_copy);
        if (s != KNN_OK) return s;
    }
    h->launches += l;
    h->searches += 1;

    if (!io_on_device) {
        if (!out_direct) {
            KNN_CUDA(h, cudaMemcpyAsync(dist_out, dd, static_cast<size_t>(n) * k * 4,
                                        cudaMemcpyDeviceToHost, st));
            KNN_CUDA(h, cudaMemcpyAsync(idx_out, id, static_cast<size_t>(n) * k * 4,
                                        cudaMemcpyDeviceToHost, st));
            stage(h, st, "d2h");
        }
        // the error flag comes back with the stream's last copy, so the one
        // synchronisation also ends the call
        KNN_CUDA(h, cudaMemcpyAsync(h->flag_host, &ctr->error_flag, sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, st));
        KNN_CUDA(h, cudaStreamSynchronize(st));
        const int32_t flag = *h->flag_host;
        if (flag) {
            KNN_CUDA(h, cudaMemset(&ctr->error_flag, 0, sizeof(flag)));
            h->last_error = "a bounded device-side wait gave up";
            return KNN_ERR_TIMEOUT;
        }
    }
    return KNN_OK;
}

knn_status knn_search_batch(knn_handle h, const knn_instance* inst, int32_t count, int32_t flags,
                            void* cuda_stream) {
    if (!h || count < 0 || (count > 0 && !inst)) return KNN_ERR_INVALID;
    h->last_stage_ns = nullptr;
    for (int32_t i = 0; i < count; ++i) {
        knn_status s = check_instance(inst[i]);
        if (s != KNN_OK) return s;
    }
    if (count == 0) return KNN_OK;
    KNN_CUDA(h, cudaSetDevice(h->device));
    cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : h->stream;

    if (flags & KNN_BATCH_NO_GRAPH) {
        // one instance after another on st, each planned as a lone search
        BatchPlan bp;
        knn_status s = plan_batch(h, inst, count, h->num_sms, &bp);
        if (s != KNN_OK) return s;
        s = ensure_workspace(h, bp.bytes);
        if (s != KNN_OK) return s;
        int l = 0;
        for (int32_t i = 0; i < count; ++i) {
            s = enqueue_instance(h, inst[i], bp, i, st, &l);
            if (s != KNN_OK) return s;
        }
        h->launches += l;
        h->searches += count;
        h->last_batch = knn_batch_info{1, h->num_sms, l, 0, 0, 0.0, 0, 0};
        return KNN_OK;
    }

    // the persistent form (every instance in one kernel launch) unless the
    // graph of per-instance launches is asked for or some instance needs it
    const bool want_persistent = !(flags & KNN_BATCH_BRANCHES) && persistent_eligible(h, inst, count);
    const uint64_t form = want_persistent ? 0x7e57ull : 0x6a0full;
    const uint64_t exact = mix64(batch_signature(h, inst, count, true), form);
    const uint64_t shape = mix64(batch_signature(h, inst, count, false), form);
    auto it = h->graphs.find(exact);
    bool fresh = false;   // built (and described in last_batch) by this call
    if (it == h->graphs.end() && want_persistent) {
        float tune_ms = 0.f;
        bool tuned_now = false;
        auto tk = h->tuned_chunks.find(shape);
        if (tk == h->tuned_chunks.end() && (flags & KNN_BATCH_AUTOTUNE)) {
            KNN_CUDA(h, cudaStreamSynchronize(st));
            std::map<uint64_t, int64_t> best;
            knn_status s = tune_persistent(h, inst, count, st, &best, &tune_ms);
            if (s != KNN_OK && s != KNN_ERR_UNSUPPORTED) return s;
            if (s == KNN_OK) {
                tk = h->tuned_chunks.emplace(shape, best).first;
                tuned_now = true;
            }
        }
        static const std::map<uint64_t, int64_t> kNone;
        knn_ctx::BatchGraph g;
        knn_status s = build_persistent(
            h, persist_inputs(inst, count, tk == h->tuned_chunks.end() ? kNone : tk->second), &g);
        if (s == KNN_OK) {
            it = h->graphs.emplace(exact, g).first;
            fresh = true;
            h->last_batch = knn_batch_info{1, h->num_sms, 1, static_cast<int64_t>(g.nodes),
                                           tuned_now ? 1 : 0, static_cast<double>(tune_ms), 1,
                                           g.pb.nitems};
        } else if (s != KNN_ERR_UNSUPPORTED) {
            return s;
        }
    }
    if (it == h->graphs.end()) {
        knn_ctx::BatchGraph best;
        float tune_ms = 0.f;
        bool tuned_now = false;
        auto tk = h->tuned.find(shape);
        if (tk != h->tuned.end()) {
            knn_status s = build_batch(h, inst, count, tk->second.first, tk->second.second, &best);
            if (s != KNN_OK) return s;
        } else if (flags & KNN_BATCH_AUTOTUNE) {
            // time every candidate configuration on this batch, keep the fastest;
            // the workspace is sized for all of them first, so that no capture
            // moves it under a graph already built
            const int shares[2] = {h->num_sms, std::max(1, h->num_sms / 4)};
            const int brs[4] = {1, 4, 8, 16};
            size_t need = 0;
            for (int si = 0; si < 2; ++si) {
                BatchPlan bp;
                knn_status s = plan_batch(h, inst, count, shares[si], &bp);
                if (s != KNN_OK) return s;
                need = std::max(need, bp.bytes);
            }
            knn_status sw = ensure_workspace(h, need);
            if (sw != KNN_OK) return sw;
            float best_ms = 0.f;
            for (int si = 0; si < 2; ++si) {
                for (int bi = 0; bi < 4; ++bi) {
                    if (bi > 0 && brs[bi] > count) continue;
                    knn_ctx::BatchGraph g;
                    knn_status s = build_batch(h, inst, count, brs[bi], shares[si], &g);
                    if (s != KNN_OK) return s;
                    KNN_CUDA(h, cudaGraphLaunch(g.exec, st));            // warm
                    KNN_CUDA(h, cudaEventRecord(h->t_ev[0], st));
                    KNN_CUDA(h, cudaGraphLaunch(g.exec, st));
                    KNN_CUDA(h, cudaGraphLaunch(g.exec, st));
                    KNN_CUDA(h, cudaEventRecord(h->t_ev[1], st));
                    KNN_CUDA(h, cudaEventSynchronize(h->t_ev[1]));
                    float ms = 0.f;
                    KNN_CUDA(h, cudaEventElapsedTime(&ms, h->t_ev[0], h->t_ev[1]));
                    ms *= 0.5f;
                    tune_ms += 3.f * ms;
                    if (!best.exec || ms < best_ms) {
                        if (best.exec) cudaGraphExecDestroy(best.exec);
                        best = g;
                        best_ms = ms;
                    } else {
                        cudaGraphExecDestroy(g.exec);
                    }
                }
            }
            h->tuned[shape] = {best.branches, best.sm_share};
            tuned_now = true;
        } else {
            const int branches = std::min<int32_t>(8, count);
            knn_status s = build_batch(h, inst, count, branches, std::max(1, h->num_sms / 4), &best);
            if (s != KNN_OK) return s;
        }
        it = h->graphs.emplace(exact, best).first;
        h->last_batch = knn_batch_info{best.branches, best.sm_share, best.launches,
                                       static_cast<int64_t>(best.nodes), tuned_now ? 1 : 0,
                                       static_cast<double>(tune_ms), 0, 0};
    } else if (!fresh) {
        const knn_ctx::BatchGraph& g = it->second;
        h->last_batch = knn_batch_info{g.branches, g.sm_share, g.launches,
                                       static_cast<int64_t>(g.nodes), 0, 0.0,
                                       g.persistent ? 1 : 0, g.persistent ? g.pb.nitems : 0};
    }
    KNN_CUDA(h, cudaGraphLaunch(it->second.exec, st));
    h->launches += it->second.launches;
    h->searches += count;
    if (it->second.persistent) {
        h->last_stage_ns = it->second.pb.stage_ns;
        h->last_stage_stream = st;
    }
    return KNN_OK;
}

knn_status knn_batch_info_get(knn_handle h, knn_batch_info* out) {
    if (!h || !out) return KNN_ERR_INVALID;
    *out = h->last_batch;
    return KNN_OK;
}

knn_status knn_batch_stage_times(knn_handle h, double* wait_ms, double* work_ms, int64_t* items) {
    if (!h || !wait_ms || !work_ms || !items) return KNN_ERR_INVALID;
    if (!h->last_stage_ns) return KNN_ERR_UNSUPPORTED;
    KNN_CUDA(h, cudaSetDevice(h->device));
    KNN_CUDA(h, cudaStreamSynchronize(h->last_stage_stream));
    unsigned long long v[3 * kPersistStages];
    KNN_CUDA(h, cudaMemcpy(v, h->last_stage_ns, sizeof(v), cudaMemcpyDeviceToHost));
    for (int s = 0; s < kPersistStages; ++s) {
        wait_ms[s] = static_cast<double>(v[s]) * 1e-6;
        work_ms[s] = static_cast<double>(v[kPersistStages + s]) * 1e-6;
        items[s] = static_cast<int64_t>(v[2 * kPersistStages + s]);
    }
    return KNN_OK;
}

knn_status knn_search_self(knn_handle h, int32_t k, knn_metric metric, float* dist_out,
                           int32_t* idx_out, void* cuda_stream) {
    if (!h || !dist_out || !idx_out) return KNN_ERR_INVALID;
    h->last_stage_ns = nullptr;
    if (!h->ref) return KNN_ERR_NOREF;
    if (k < 1 || static_cast<int64_t>(k) + 1 > h->ref->m) return KNN_ERR_INVALID;
    knn_status s = check_search_args(h, h->ref->m, h->ref->d, k + 1, metric);
    if (s != KNN_OK) return s;
    if (metric == KNN_MAHALANOBIS) return KNN_ERR_UNSUPPORTED;
    KNN_CUDA(h, cudaSetDevice(h->device));
    cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : h->stream;
    RefSet& rs = *h->ref;
    const int64_t n = rs.m;
    SearchPlan sp;
    s = plan_search(h, n, k + 1, metric, 1, &sp);
    if (s != KNN_OK) return s;
    if (sp.tensor) {
        s = build_lowp(h, sp.prec);
        if (s != KNN_OK) return s;
    }
    // the (k+1)-neighbour rows go to workspace after the search's own slices
    Carve cv;
    cv.off = sp.bytes;
    const size_t off_d = cv.take(static_cast<size_t>(n) * (k + 1) * sizeof(float));
    const size_t off_i = cv.take(static_cast<size_t>(n) * (k + 1) * sizeof(int32_t));
    s = ensure_workspace(h, cv.off);
    if (s != KNN_OK) return s;
    unsigned char* ws = h->ws;
    float* dtmp = reinterpret_cast<float*>(ws + off_d);
    int32_t* itmp = reinterpret_cast<int32_t*>(ws + off_i);
    int l = 0;
    h->nstages = 0;
    RefView rv{rs.R, rs.m, rs.d, rs.R_lp, rs.kp, rs.rmax2};
    s = enqueue_search(h, sp, rv, rs.R, n, k + 1, metric, dtmp, itmp, ws, &h->counters->fallback_count,
                       st, &l, false);
    if (s != KNN_OK) return s;
    KNN_CUDA(h, launch_drop_self(dtmp, itmp, n, k, dist_out, idx_out, st, &l));
    h->launches += l;
    h->searches += 1;
    return KNN_OK;
}

knn_status knn_sync(knn_handle h) {
    if (!h) return KNN_ERR_INVALID;
    KNN_CUDA(h, cudaSetDevice(h->device));
    KNN_CUDA(h, cudaDeviceSynchronize());
    int32_t flag = 0;
    KNN_CUDA(h, cudaMemcpy(&flag, &h->counters->error_flag, sizeof(flag), cudaMemcpyDeviceToHost));
    if (flag) {
        KNN_CUDA(h, cudaMemset(&h->counters->error_flag, 0, sizeof(flag)));
        h->last_error = "a bounded device-side wait gave up";
        return KNN_ERR_TIMEOUT;
    }
    return KNN_OK;
}

knn_status knn_explain_plan(int64_t n, int64_t m, int32_t d, int32_t k, knn_metric metric,
                            int32_t precision, int32_t rerank_factor, int32_t num_sms,
                            knn_plan* out) {
    if (!out || n < 1 || m < 1 || d < 1 || k < 1 || k > m || num_sms < 1) return KNN_ERR_INVALID;
    if (metric != KNN_L2 && metric != KNN_L1 && metric != KNN_LINF && metric != KNN_MAHALANOBIS)
        return KNN_ERR_INVALID;
    if (precision < KNN_FP32 || precision > KNN_BF16 || rerank_factor < 1 || rerank_factor > 64)
        return KNN_ERR_INVALID;
    if (k > KNN_K_MAX || m > 0x7fffffffLL || n > 0x7fffffffLL) return KNN_ERR_UNSUPPORTED;
    knn_ctx h;   // only its options are read by the planner
    h.opt.rerank_factor = rerank_factor;
    h.opt.precision = precision;
    SearchPlan sp;
    const knn_metric planned = metric == KNN_MAHALANOBIS ? KNN_L2 : metric;
    knn_status s = plan_search_md(&h, m, d, precision, n, k, planned, 1, num_sms, &sp);
    if (s != KNN_OK) return s;
    knn_plan o{};
    o.tensor_cores = sp.tensor ? 1 : 0;
    o.candidates = sp.c;
    o.splits = sp.S;
    o.chunk = sp.chunk;
    if (sp.tensor) {
        o.k_blocks = sp.plan.kb;
        o.stages = sp.plan.stages;
        o.whole_tile_stages = sp.plan.kbs == sp.plan.kb ? 1 : 0;
        o.raw_staging = sp.plan.raw;
        o.pilot = sp.plan.pilot;
        o.pilot_stride = sp.plan.stride;
        o.pilot_groups = sp.plan.G;
        o.pilot_group_size = sp.plan.gsize;
        o.threshold_rank = sp.plan.cprime;
        o.list_capacity = sp.plan.cap;
    }
    o.fallback_slots = static_cast<int32_t>(sp.fb_grid);
    o.workspace_bytes = static_cast<int64_t>(sp.bytes);
    o.small_select = sp.small ? 1 : 0;
    *out = o;
    return KNN_OK;
}

knn_status knn_selftest_bounded_wait(knn_handle h, int32_t limit_ms) {
    if (!h || limit_ms < 1 || limit_ms > 1000) return KNN_ERR_INVALID;
    KNN_CUDA(h, cudaSetDevice(h->device));
    KNN_CUDA(h, launch_wait_probe(&h->counters->error_flag,
                                  static_cast<uint64_t>(limit_ms) * 1000000ull, h->stream));
    return knn_sync(h);
}

knn_status knn_selftest_batch_queue(knn_handle h, int32_t limit_ms) {
    if (!h || limit_ms < 1 || limit_ms > 1000) return KNN_ERR_INVALID;
    KNN_CUDA(h, cudaSetDevice(h->device));
    KNN_CUDA(h, cudaStreamSynchronize(h->stream));
    // a one-instance batch (64 points in d = 32) whose buffers the kernel never
    // reaches: every CTA gives up at the withheld ready word
    constexpr int64_t n = 64;
    constexpr int32_t d = 32, k = 4;
    unsigned char* buf = nullptr;
    const size_t pts = static_cast<size_t>(n) * d * sizeof(float);
    const size_t outs = static_cast<size_t>(n) * k * sizeof(float);
    KNN_CUDA(h, cudaMalloc(&buf, 2 * pts + 2 * outs));
    const float* R = reinterpret_cast<const float*>(buf);
    const float* Q = reinterpret_cast<const float*>(buf + pts);
    float* dist = reinterpret_cast<float*>(buf + 2 * pts);
    int32_t* idx = reinterpret_cast<int32_t*>(buf + 2 * pts + outs);
    const std::vector<PersistInst> pin{PersistInst{R, n, Q, n, d, k, dist, idx, 0}};
    PersistPlan pp;
    PersistBatch pb;
    knn_status s = KNN_OK;
    cudaError_t err = persist_plan(pin, kBF16, h->opt.rerank_factor, h->num_sms, &pp);
    if (err != cudaSuccess) s = cuda_fail(h, err, "persist_plan");
    if (s == KNN_OK) s = ensure_workspace(h, pp.ws_bytes);
    if (s == KNN_OK) {
        PersistCounters ctr{&h->counters->error_flag, &h->counters->recheck_total,
                            &h->counters->fallback_total, h->counters->fallback_reason};
        err = persist_build(pin, pp, kBF16, h->ws, ctr, &pb);
        if (err == cudaSuccess)
            err = persist_launch(pb, h->num_sms, false, static_cast<uint64_t>(limit_ms) * 1000000ull,
                                 h->stream);
        if (err != cudaSuccess) s = cuda_fail(h, err, "persistent batch self-test");
    }
    if (s == KNN_OK) s = knn_sync(h);
    else cudaDeviceSynchronize();
    persist_free(&pb);
    cudaFree(buf);
    return s;
}

knn_status knn_get_stats(knn_handle h, knn_stats* out) {
    if (!h || !out) return KNN_ERR_INVALID;
    KNN_CUDA(h, cudaSetDevice(h->device));
    KNN_CUDA(h, cudaDeviceSynchronize());
    Counters c{};
    KNN_CUDA(h, cudaMemcpy(&c, h->counters, sizeof(c), cudaMemcpyDeviceToHost));
    out->searches = h->searches;
    out->kernel_launches = h->launches;
    out->recheck_entries = static_cast<int64_t>(c.recheck_total);
    out->fallback_queries = static_cast<int64_t>(c.fallback_total);
    out->workspace_bytes = static_cast<int64_t>(h->ws_bytes);
    out->fallback_short_list = static_cast<int64_t>(c.fallback_reason[0]);
    out->fallback_overflow = static_cast<int64_t>(c.fallback_reason[1]);
    out->fallback_wide_cut = static_cast<int64_t>(c.fallback_reason[2]);
    out->fallback_uncertified = static_cast<int64_t>(c.fallback_reason[3]);
    return KNN_OK;
}

knn_status knn_set_profiling(knn_handle h, int on) {
    if (!h) return KNN_ERR_INVALID;
    h->profiling = on != 0;
    h->nstages = 0;
    return KNN_OK;
}

knn_status knn_get_profile(knn_handle h, float* ms, const char** names, int32_t cap,
                           int32_t* count) {
    if (!h || !count || cap < 0 || (cap > 0 && (!ms || !names))) return KNN_ERR_INVALID;
    KNN_CUDA(h, cudaSetDevice(h->device));
    const int ns = h->nstages;
    if (ns > 0) KNN_CUDA(h, cudaEventSynchronize(h->ev[ns]));
    for (int i = 0; i < ns && i < cap; ++i) {
        float t = 0.f;
        KNN_CUDA(h, cudaEventElapsedTime(&t, h->ev[i], h->ev[i + 1]));
        ms[i] = t;
        names[i] = h->stage_names[i];
    }
    *count = ns;
    return KNN_OK;
}

const char* knn_status_string(knn_status s) {
    switch (s) {
        case KNN_OK: return "ok";
        case KNN_ERR_INVALID: return "invalid argument";
        case KNN_ERR_OOM: return "out of device memory";
        case KNN_ERR_CUDA: return "CUDA error";
        case KNN_ERR_TIMEOUT: return "device wait timed out";
        case KNN_ERR_NOREF: return "no reference set";
        case KNN_ERR_BUSY: return "reference set or handle busy";
        case KNN_ERR_UNSUPPORTED: return "unsupported by this build";
    }
    return "unknown status";
}

const char* knn_last_error(knn_handle h) { return h ? h->last_error.c_str() : ""; }

}  // extern "C"
