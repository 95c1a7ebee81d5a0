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
// staged in shared memory; a block takes 32 rows, one thread per (row, output
// coordinate) pair.
#include "knn_internal.cuh"

namespace knn {
namespace {

constexpr int kRowsPerBlock = 32;
constexpr int kThreads = 256;

// a + b as an unevaluated pair (hi, lo) with hi = fl(a + b) (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float& hi, float& lo) {
    hi = a + b;
    const float bb = hi - a;
    lo = (a - (hi - bb)) + (b - bb);
}

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
    for (int t = threadIdx.x; t < nr * d; t += blockDim.x) {
        const int row = t / d, j = t % d;
        const float* x = sX + row * d;
        float hi = 0.f, lo = 0.f;
        for (int i = j; i < d; ++i) {
            const float a = x[i], b = sL[i * d + j];
            const float p = a * b;
            const float e = fmaf(a, b, -p);                  // a * b = p + e exactly
            float s, c;
            two_sum(hi, p, s, c);
            hi = s;
            lo += c + e;
        }
        Y[(r0 + row) * d + j] = hi + lo;
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
    cudaError_t err = cudaFuncSetAttribute(whiten_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    const unsigned grid = static_cast<unsigned>((rows + kRowsPerBlock - 1) / kRowsPerBlock);
    whiten_kernel<<<grid, kThreads, smem, st>>>(X, rows, d, L, Y);
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace knn
