// knn_internal.cuh -- declarations shared by the kernel files of the library.
//
// The search (Sec. 2.1 of Garcia, Debreuve, Barlaud, "Fast k Nearest Neighbor
// Search using GPU") runs as three stages, all on the GPU:
//   1. select   -- a fused distance + per-query top-c kernel: each tile of the
//                  n x m distance matrix is produced on chip and consumed at
//                  once by a per-query selection; only c candidates per query
//                  (and per reference split) reach global memory.  The CUDA-core
//                  form (knn_cc.cu) computes float32 distances from coordinate
//                  differences; the tensor-core form (knn_tc.cu) computes the
//                  cross term q.r with tcgen05 and ranks by ||r||^2 - 2 q.r.
//   2. finalize -- per query: exact float32 distances of the candidates, a sort
//                  by (distance, index), a float64 re-check of candidates whose
//                  float32 distances are within rounding of each other, and the
//                  k outputs (knn_finalize.cu).  Queries whose candidate set
//                  cannot be certified complete are queued for stage 3.
//   3. fallback -- exact float64 distances to every reference and an exact
//                  radix selection, for the queued queries only (rare: it needs
//                  more near-equal distances than there are spare candidates).
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

namespace knn {

// Opt kernel KERN in to `smem` bytes of dynamic shared memory, once per
// device and size: cudaFuncSetAttribute costs host time on every call (tens
// of microseconds in front of an idle GPU), and the setting persists.
template <auto KERN>
cudaError_t allow_smem(size_t smem) {
    constexpr int kDevs = 64;
    static std::atomic<size_t> done[kDevs];
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    const bool tracked = dev >= 0 && dev < kDevs;
    if (tracked && smem <= done[dev].load(std::memory_order_relaxed)) return cudaSuccess;
    err = cudaFuncSetAttribute(KERN, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err == cudaSuccess && tracked) {
        size_t cur = done[dev].load(std::memory_order_relaxed);
        while (smem > cur && !done[dev].compare_exchange_weak(cur, smem)) {
        }
    }
    return err;
}

enum Metric : int { kL2 = 0, kL1 = 1, kLinf = 2 };

constexpr uint64_t kEmptyKey = ~0ull;  // sentinel for an empty candidate slot

// Order-preserving map float -> uint32 (total order on non-NaN floats).
__host__ __device__ __forceinline__ uint32_t ord_f32(float x) {
#ifdef __CUDA_ARCH__
    uint32_t b = __float_as_uint(x);
#else
    uint32_t b;
    __builtin_memcpy(&b, &x, 4);
#endif
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__host__ __device__ __forceinline__ float unord_f32(uint32_t o) {
    uint32_t b = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float x;
    __builtin_memcpy(&x, &b, 4);
    return x;
#endif
}

// Candidate key: (distance, index) packed so that unsigned comparison is the
// lexicographic order of the pair (smaller distance first, then smaller index).
__host__ __device__ __forceinline__ uint64_t make_key(float dist, uint32_t idx) {
    return (static_cast<uint64_t>(ord_f32(dist)) << 32) | idx;
}
__host__ __device__ __forceinline__ uint32_t key_idx(uint64_t key) {
    return static_cast<uint32_t>(key & 0xffffffffu);
}
__host__ __device__ __forceinline__ float key_dist(uint64_t key) {
    return unord_f32(static_cast<uint32_t>(key >> 32));
}

// Where the candidates of one search live: n queries x S reference splits x c.
// Split s covers references [s*chunk, min(m, (s+1)*chunk)).
struct CandidateSet {
    uint64_t* keys;   // [n][S][c]
    int64_t n;
    int32_t S;
    int32_t c;
    int64_t chunk;
    int32_t exact;    // 1: key distances are float32 distances of the metric
                      //    (completeness can be certified); 0: ranking scores
};

// Per-query lists of references that passed the tensor-core filter (S lists
// per query: one per reference split and epilogue column group).  A key is
// (code, index) with code in [0, 0xffff] falling linearly with the
// low-precision score (smaller code = nearer).  counts may exceed cap,
// meaning the list overflowed.
struct HitLists {
    const uint64_t* keys;   // [n][S][cap]
    const int32_t* counts;  // [n][S]
    int32_t S;
    int32_t cap;
    int32_t c;              // keep (at least) the best c before the exact re-rank
};

struct FinalizeArgs {
    int32_t use_hits;       // 0: candidates come from `cand`; 1: from `hits`
    HitLists hits;
    const float* Q;
    const float* R;
    int64_t n, m;
    int32_t d, k;
    int32_t metric;
    CandidateSet cand;
    float* dist_out;
    int32_t* idx_out;
    int32_t* fallback_count;   // device counter of queued queries
    int32_t* fallback_list;    // [n] query ids
    unsigned long long* recheck_counter;
    unsigned long long* fallback_total;
    unsigned long long* fallback_reason;   // [4]: short list, overflow, wide cut, uncertified
    int32_t* fb_done;                      // fallback chunk counters to zero, or null
    int32_t fb_slots;
    // rounding bounds for this d, set by launch_finalize: float32 distance
    // (relative), its near-tie window as a float, and the float-float window
    double rel;
    float relf;
    float ffw;
};

// ---- launchers (return cudaSuccess or the launch error) -------------------

// CUDA-core fused distance + top-c.  Writes cand (exact = 1).
cudaError_t launch_cc_select(const float* Q, int64_t n, const float* R, int64_t m, int32_t d,
                             int32_t metric, const CandidateSet& cand, cudaStream_t st,
                             int* launches);

// The largest c launch_cc_select supports.
int cc_max_candidates();

// Float32 select for small reference sets (knn_small.cu): one warp per query
// holds all m distances in shared memory and selects exactly a set of keys
// that holds its c_need nearest and that no key left out precedes, of at most
// cand.c (>= c_need) keys, the unused slots empty.  Writes cand with S = 1
// split of the whole set (exact = 1).  Available when small_select_fits(m, d):
// m up to kSmallSelectMaxM and the shared memory (small_select_smem) within
// one CTA's.  kSmallSelectSpare: the spare slots a search plans beyond c_need.
constexpr int64_t kSmallSelectMaxM = 4096;
constexpr int kSmallSelectSpare = 16;
// Tensor-core searches whose pilot runs still take the small-set select while
// ceil(n / 8) * m * d / SMs (an SM's share of its distance products) is below this.
constexpr double kSmallSelectShare = 2.2e5;
size_t small_select_smem(int64_t m, int32_t d);
bool small_select_fits(int64_t m, int32_t d);
cudaError_t launch_small_select(const float* Q, int64_t n, const float* R, int64_t m, int32_t d,
                                int32_t metric, int32_t c_need, const CandidateSet& cand,
                                cudaStream_t st, int* launches);

// Reference splits S of the float32 search and their length *chunk (a
// multiple of 128): among the S with every split at least 8c long and S*c
// within max_pool, and at least two CTAs per SM where that is possible, the
// one with the least estimated time, the CTAs resident on an SM sharing its
// throughput (so a partly filled last wave of CTAs costs what its busiest SM
// holds).
int cc_plan_splits(int64_t n, int64_t m, int32_t c, int num_sms, int max_pool, int64_t* chunk);

cudaError_t launch_finalize(const FinalizeArgs& a, cudaStream_t st, int* launches);
int finalize_max_pool();   // largest S*c one finalize pass handles

// Whitening for the Mahalanobis distance (knn_whiten.cu): Y = X L for rows
// of X (rows x d), L the d x d lower-triangular Cholesky factor of the inverse
// covariance (row-major float32); compensated accumulation, one rounding.
size_t whiten_smem_bytes(int32_t d);
cudaError_t launch_whiten(const float* X, int64_t rows, int32_t d, const float* L, float* Y,
                          cudaStream_t st, int* launches);

// One bounded mbarrier wait that nothing completes: raises *error_flag after
// limit_ns (the failure path of every device-side wait, exercised on purpose).
cudaError_t launch_wait_probe(int32_t* error_flag, uint64_t limit_ns, cudaStream_t st);

// Self-join rows: the n x (k+1) result of searching R against itself, minus
// each row's own index (or its last entry), into n x k outputs.
cudaError_t launch_drop_self(const float* din, const int32_t* iin, int64_t n, int32_t k, float* dout,
                             int32_t* iout, cudaStream_t st, int* launches);

// Exact float64 pass for the queued queries.  scratch holds slots*m doubles;
// done holds `slots` counters, zeroed by the finalize that runs before (its
// FinalizeArgs::fb_done / fb_slots).  The first slots/2 queued queries have
// their float32 key pass spread over the GPU; the rest take one CTA each.
cudaError_t launch_fallback(const FinalizeArgs& a, double* scratch, int32_t slots, int32_t* done,
                            cudaStream_t st, int* launches);

// ---- tensor-core path (knn_tc.cu) -----------------------------------------

enum LowPrecision : int { kTF32 = 1, kBF16 = 2 };

// Row length (elements) of the low-precision operand copies: d coordinates,
// four augmentation words (norm halves, threshold halves), zero padded to a
// whole number of 128-byte K blocks.
int tc_padded_dim(int32_t d, int prec);

// Launch plan of the pilot and filter passes for one search.
struct TcPlan {
    int32_t mt;          // 128-query tiles per CTA (1)
    int32_t kb;          // 128-byte K blocks per operand row
    int32_t ksteps;      // 32-byte MMA K steps that carry data
    int32_t rb;          // references per tile (MMA N = 256)
    int32_t kbs;         // K blocks per TMA stage (kb, or 1 for long rows)
    int32_t groups;      // hit lists per (query, split): one per epilogue column group
    int32_t stages;      // reference-stage ring depth
    int32_t S;           // reference splits
    int64_t chunk;       // references per split (multiple of rb)
    int32_t stride;      // pilot samples every stride-th stage
    int32_t spt;         // pilot tile slots per split
    int32_t G;           // pilot group maxima per query
    int32_t gsize;       // references per pilot group (32, or 16 / 8 when every tile is sampled)
    int32_t cprime;      // order statistic of the group maxima used as threshold
    int32_t pilot;       // 0: no pilot, every reference is appended
    int32_t cap;         // list capacity per (query, split, column group)
    int32_t raw;         // filter stages hit values as float32 (else 16-bit codes)
    size_t smem_filter;
};
// smem_limit: the dynamic shared memory an item may use (the persistent batch
// kernel keeps some for itself); force_chunk > 0: split the references into
// pieces of about this length (rounded to whole tiles) instead of choosing the
// split count by how full the last wave of CTAs is.
TcPlan tc_plan(int64_t n, int64_t m, int32_t d, int32_t kp, int prec, int32_t c, int num_sms,
               size_t smem_limit = 232448, int64_t force_chunk = 0);

// Per-query scale of the 16-bit hit codes (a power of two B > |acc|): the
// largest squared reference norm (float bits, set by launch_prepare_ref) and
// the queries' B, set by launch_tc_threshold once t is known, or by
// launch_prepare_query for t = 0 when qscale is passed there (no threshold).
struct HitScale {
    const uint32_t* rmax2;
    float* qscale;   // [n]
};

// Reference copy [r, -||r||^2/2 (hi, lo), 1, 1, 0..], float32 norms and their maximum.
cudaError_t launch_prepare_ref(const float* R, int64_t m, int32_t d, int32_t kp, int prec,
                               void* R_lp, float* norms, uint32_t* rmax2, cudaStream_t st,
                               int* launches);
// Query copy [q, 1, 1, 0, 0, 0..] (threshold words filled by the threshold pass);
// when Q_copy is given, the float32 rows are also written there (Q may then be
// host memory the GPU reads directly).
cudaError_t launch_prepare_query(const float* Q, int64_t n, int32_t d, int32_t kp, int prec,
                                 void* Q_lp, const HitScale& qs, float* Q_copy, cudaStream_t st,
                                 int* launches);
cudaError_t launch_tc_pilot(const TcPlan& p, const void* Q_lp, int64_t n, const void* R_lp,
                            int64_t m, int32_t kp, int prec, uint32_t* gmax, int32_t* error_flag,
                            cudaStream_t st, int* launches);
cudaError_t launch_tc_threshold(const TcPlan& p, const uint32_t* gmax, int64_t n, int32_t d,
                                int32_t kp, int prec, void* Q_lp, const HitScale& qs,
                                cudaStream_t st, int* launches);
cudaError_t launch_tc_filter(const TcPlan& p, const void* Q_lp, int64_t n, const void* R_lp,
                             int64_t m, int32_t kp, int prec, uint64_t* lists, int32_t* counts,
                             const float* qscale, int32_t* error_flag, cudaStream_t st,
                             int* launches);

}  // namespace knn
