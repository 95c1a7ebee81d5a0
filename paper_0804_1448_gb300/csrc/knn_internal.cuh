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

#include <cstdint>
#include <cuda_runtime.h>

namespace knn {

enum Metric : int { kL2 = 0, kL1 = 1 };

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

struct FinalizeArgs {
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
};

// ---- launchers (return cudaSuccess or the launch error) -------------------

// CUDA-core fused distance + top-c.  Writes cand (exact = 1).
cudaError_t launch_cc_select(const float* Q, int64_t n, const float* R, int64_t m, int32_t d,
                             int32_t metric, const CandidateSet& cand, cudaStream_t st,
                             int* launches);

// Bytes of dynamic shared memory launch_cc_select needs for c candidates,
// and the largest c it supports.
int cc_max_candidates();

cudaError_t launch_finalize(const FinalizeArgs& a, cudaStream_t st, int* launches);
int finalize_max_pool();   // largest S*c one finalize pass handles

// Exact float64 pass for the queued queries.  scratch holds grid*m doubles.
cudaError_t launch_fallback(const FinalizeArgs& a, double* scratch, int32_t grid,
                            cudaStream_t st, int* launches);

// ---- tensor-core path (knn_tc.cu) -----------------------------------------

enum LowPrecision : int { kTF32 = 1, kBF16 = 2 };

// Build the low-precision operand copy of a point set: rows of `kp` elements
// (bf16 or tf32-in-fp32), zero padded beyond d, plus the float32 squared
// norms of the float32 rows (norms may be NULL).
cudaError_t launch_prepare_lowp(const float* X, int64_t rows, int32_t d, int32_t kp, int prec,
                                void* X_lp, float* norms, cudaStream_t st, int* launches);
int tc_padded_dim(int32_t d, int prec);
// Largest candidate count per query the tensor-core kernel holds on chip.
int tc_max_candidates(int32_t kp, int prec);
// Tensor-core fused q.r + top-c.  Writes cand (exact = 0).
cudaError_t launch_tc_select(const void* Q_lp, int64_t n, const void* R_lp, const float* r_norms,
                             int64_t m, int32_t kp, int prec, const CandidateSet& cand,
                             int32_t* error_flag, cudaStream_t st, int* launches);

}  // namespace knn
