// knn_whiten.cu -- the whitening transform behind the Mahalanobis distance.
//
// Sec. 2.1 of the paper admits any distance besides the Euclidean and
// Manhattan ones and names the Mahalanobis distance
//     d_M(q, r)^2 = (q - r)^T S^-1 (q - r)
// for a covariance S.  With the Cholesky factor of the inverse covariance,
// S^-1 = L L^T (L lower triangular), d_M(q, r) = || L^T q - L^T r ||_2, so the
// search runs as a Euclidean search over whitened points x' = L^T x: every
// form of the Euclidean path (float32 CUDA cores, bf16 / tf32 tensor cores,
// the float32 re-rank and the near-tie tiers) applies unchanged.
//
// whiten_kernel computes x'_j = sum_{i >= j} x_i L[i][j] for every row with
// the compensated dot product "Dot2" of Ogita, Rump and Oishi (2005): each
// product split exactly by a fused multiply-add, the running sum by Knuth's
// two-sum, the error terms summed aside and added once at the end, so each
// whitened coordinate is as accurate as if computed in twice the working
// precision and then rounded to float32.  L (d x d, row-major, float32) is
// staged in shared memory; a block takes 32 rows, each thread four rows and
// every 32nd output coordinate.
#include "knn_internal.cuh"

namespace knn {
namespace {

constexpr int kRowsPerBlock = 32;
constexpr int kThreads = 256;
constexpr int kRowsPerWarp = kRowsPerBlock / (kThreads / 32);   // 4

// a + b as an unevaluated pair (hi, lo) with hi = fl(a + b) (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float& hi, float& lo) {
    hi = a + b;
    const float bb = hi - a;
    lo = (a - (hi - bb)) + (b - bb);
}

// One Dot2 step: (hi, lo) += a * b, the product split exactly by an FMA.
__device__ __forceinline__ void dot2_step(float a, float b, float& hi, float& lo) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    float s, c;
    two_sum(hi, p, s, c);
    hi = s;
    lo += c + e;
}

// Warp w takes rows 4w..4w+3 of the block's 32; lane l the output coordinates
// j = l + 32 c (c < NJ = ceil(d / 32)): 4 NJ independent compensated sums per
// thread, advanced together over i (a term exists when i >= j).
template <int NJ>
__global__ void __launch_bounds__(kThreads)
whiten_kernel(const float* __restrict__ X, int64_t rows, int32_t d, const float* __restrict__ L,
              float* __restrict__ Y) {
    extern __shared__ float sm[];
    float* sL = sm;                                          // d x d
    float* sX = sm + static_cast<size_t>(d) * d;             // kRowsPerBlock x d
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kRowsPerBlock;
    const int nr = static_cast<int>(min(static_cast<int64_t>(kRowsPerBlock), rows - r0));
    for (int t = threadIdx.x; t < d * d; t += blockDim.x) sL[t] = L[t];
    for (int t = threadIdx.x; t < nr * d; t += blockDim.x) sX[t] = X[r0 * d + t];
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int rb = warp * kRowsPerWarp;
    float hi[kRowsPerWarp][NJ], lo[kRowsPerWarp][NJ];
#pragma unroll
    for (int r = 0; r < kRowsPerWarp; ++r)
#pragma unroll
        for (int c = 0; c < NJ; ++c) hi[r][c] = lo[r][c] = 0.f;
    for (int i = 0; i < d; ++i) {
        float x[kRowsPerWarp];
#pragma unroll
        for (int r = 0; r < kRowsPerWarp; ++r) x[r] = (rb + r < nr) ? sX[(rb + r) * d + i] : 0.f;
#pragma unroll
        for (int c = 0; c < NJ; ++c) {
            const int j = lane + 32 * c;
            if (j <= i) {                                    // L[i][j] = 0 above the diagonal
                const float b = sL[i * d + j];
#pragma unroll
                for (int r = 0; r < kRowsPerWarp; ++r) dot2_step(x[r], b, hi[r][c], lo[r][c]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kRowsPerWarp; ++r)
#pragma unroll
        for (int c = 0; c < NJ; ++c) {
            const int j = lane + 32 * c;
            if (rb + r < nr && j < d) Y[(r0 + rb + r) * d + j] = hi[r][c] + lo[r][c];
        }
}

}  // namespace

size_t whiten_smem_bytes(int32_t d) {
    return (static_cast<size_t>(d) * d + static_cast<size_t>(kRowsPerBlock) * d) * sizeof(float);
}

cudaError_t launch_whiten(const float* X, int64_t rows, int32_t d, const float* L, float* Y,
                          cudaStream_t st, int* launches) {
    if (rows <= 0) return cudaSuccess;
    const size_t smem = whiten_smem_bytes(d);
    if (d > 224) return cudaErrorInvalidValue;
    const unsigned grid = static_cast<unsigned>((rows + kRowsPerBlock - 1) / kRowsPerBlock);
    cudaError_t err = cudaSuccess;
    switch ((d + 31) / 32) {
#define KNN_WHITEN_CASE(NJ)                                                          \
        case NJ:                                                                     \
            err = allow_smem<whiten_kernel<NJ>>(smem);                              \
            if (err == cudaSuccess) whiten_kernel<NJ><<<grid, kThreads, smem, st>>>(X, rows, d, L, Y); \
            break;
        KNN_WHITEN_CASE(1) KNN_WHITEN_CASE(2) KNN_WHITEN_CASE(3) KNN_WHITEN_CASE(4)
        KNN_WHITEN_CASE(5) KNN_WHITEN_CASE(6)
        default: KNN_WHITEN_CASE(7)
#undef KNN_WHITEN_CASE
    }
    if (err != cudaSuccess) return err;
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace knn
