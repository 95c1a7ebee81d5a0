// knn_cc.cu -- float32 CUDA-core fused distance + per-query top-c selection.
//
// Step 1 of the brute-force algorithm of Sec. 2.1 (all distances between q_i
// and the r_j) fused with steps 2-3 (sort, keep the smallest): a CTA owns
// ROWS queries and streams the references of its split through shared memory
// in tiles of TM; each thread accumulates an RR x CN register micro-tile of
// distances over the d coordinates; the finished tile goes to shared memory and
// one thread per query pushes it through that query's bounded max-heap of c
// candidates.  Only the c survivors per (query, split) are written out.
//
// Distances are formed from coordinate differences in float32, coordinate 0
// first: Euclidean sum_t fma(q_t - r_t, q_t - r_t, acc) (the squared
// distance), Manhattan sum_t |q_t - r_t|.  Nothing is expanded, so a query
// that equals a reference gets exactly 0.
#include "knn_internal.cuh"

namespace knn {
namespace {

constexpr int kThreads = 256;
constexpr int kDK = 16;    // coordinates per shared-memory stage
constexpr int kTM = 128;   // references per tile

template <int ROWS>
struct CCShape;
template <>
struct CCShape<64> {       // 16 x 16 threads, 4 queries x 8 references each
    static constexpr int TY = 16, TX = 16, RR = 4, CN = 8, G = 4;
};
template <>
struct CCShape<16> {       // 4 x 64 threads, 4 queries x 2 references each
    static constexpr int TY = 4, TX = 64, RR = 4, CN = 2, G = 2;
};

template <int ROWS>
constexpr size_t cc_smem_bytes(int c) {
    return sizeof(float) * (kDK * (ROWS + 4) + kDK * (kTM + 4) + ROWS * (kTM + 1)) +
           sizeof(uint64_t) * static_cast<size_t>(c) * ROWS;
}

// Max-heap (largest key at slot 0) of c keys, slot-major with stride ROWS.
// Replace the top by `key` (key < top) and sift down.
template <int ROWS>
__device__ __forceinline__ void heap_replace_top(uint64_t* h, int c, uint64_t key) {
    int i = 0;
    while (true) {
        int l = 2 * i + 1;
        if (l >= c) break;
        uint64_t big = h[l * ROWS];
        int bi = l;
        if (l + 1 < c) {
            uint64_t rv = h[(l + 1) * ROWS];
            if (rv > big) { big = rv; bi = l + 1; }
        }
        if (big <= key) break;
        h[i * ROWS] = big;
        i = bi;
    }
    h[i * ROWS] = key;
}

template <int METRIC, int ROWS>
__global__ void __launch_bounds__(kThreads)
cc_select_kernel(const float* __restrict__ Q, int64_t n, const float* __restrict__ R,
                 int64_t m, int32_t d, CandidateSet cand) {
    using S = CCShape<ROWS>;
    static_assert(S::TY * S::TX == kThreads, "thread shape");
    static_assert(S::TY * S::RR == ROWS && S::TX * S::CN == kTM, "tile shape");
    constexpr int QST = ROWS + 4;      // padded strides (bank spread)
    constexpr int RST = kTM + 4;
    constexpr int DST = kTM + 1;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Qs = reinterpret_cast<float*>(smem_raw);            // [kDK][QST]
    float* Rs = Qs + kDK * QST;                                // [kDK][RST]
    float* Dt = Rs + kDK * RST;                                // [ROWS][DST]
    uint64_t* heap = reinterpret_cast<uint64_t*>(Dt + ROWS * DST);  // [c][ROWS]

    const int tid = threadIdx.x;
    const int ty = tid / S::TX, tx = tid % S::TX;
    const int c = cand.c;
    const int64_t qbase = static_cast<int64_t>(blockIdx.x) * ROWS;
    const int split = blockIdx.y;
    const int64_t r_begin = static_cast<int64_t>(split) * cand.chunk;
    const int64_t r_end = min(m, r_begin + cand.chunk);

    for (int e = tid; e < c * ROWS; e += kThreads) heap[e] = kEmptyKey;
    uint64_t top = kEmptyKey;  // cached heap[0] of this thread's row (selector threads)

    for (int64_t tbase = r_begin; tbase < r_end; tbase += kTM) {
        float acc[S::RR][S::CN];
#pragma unroll
        for (int i = 0; i < S::RR; ++i)
#pragma unroll
            for (int j = 0; j < S::CN; ++j) acc[i][j] = 0.f;

        for (int dbase = 0; dbase < d; dbase += kDK) {
            __syncthreads();
            for (int e = tid; e < ROWS * kDK; e += kThreads) {
                int r = e / kDK, t = e % kDK;
                int64_t gq = qbase + r;
                int gt = dbase + t;
                Qs[t * QST + r] = (gq < n && gt < d) ? Q[gq * d + gt] : 0.f;
            }
            for (int e = tid; e < kTM * kDK; e += kThreads) {
                int r = e / kDK, t = e % kDK;
                int64_t gr = tbase + r;
                int gt = dbase + t;
                Rs[t * RST + r] = (gr < r_end && gt < d) ? R[gr * d + gt] : 0.f;
            }
            __syncthreads();
#pragma unroll 4
            for (int t = 0; t < kDK; ++t) {
                float qv[S::RR], rv[S::CN];
                const float4 q4 = *reinterpret_cast<const float4*>(&Qs[t * QST + ty * S::RR]);
                qv[0] = q4.x; qv[1] = q4.y; qv[2] = q4.z; qv[3] = q4.w;
#pragma unroll
                for (int g = 0; g < S::CN / S::G; ++g) {
                    const float* src = &Rs[t * RST + g * S::TX * S::G + tx * S::G];
                    if constexpr (S::G == 4) {
                        const float4 r4 = *reinterpret_cast<const float4*>(src);
                        rv[g * 4 + 0] = r4.x; rv[g * 4 + 1] = r4.y;
                        rv[g * 4 + 2] = r4.z; rv[g * 4 + 3] = r4.w;
                    } else {
                        const float2 r2 = *reinterpret_cast<const float2*>(src);
                        rv[g * 2 + 0] = r2.x; rv[g * 2 + 1] = r2.y;
                    }
                }
#pragma unroll
                for (int i = 0; i < S::RR; ++i)
#pragma unroll
                    for (int j = 0; j < S::CN; ++j) {
                        const float diff = qv[i] - rv[j];
                        if (METRIC == kL2) acc[i][j] = fmaf(diff, diff, acc[i][j]);
                        else if (METRIC == kL1) acc[i][j] += fabsf(diff);
                        else acc[i][j] = fmaxf(acc[i][j], fabsf(diff));
                    }
            }
        }
        // tile of distances -> shared memory
#pragma unroll
        for (int i = 0; i < S::RR; ++i)
#pragma unroll
            for (int j = 0; j < S::CN; ++j) {
                const int col = (j / S::G) * (S::TX * S::G) + tx * S::G + (j % S::G);
                Dt[(ty * S::RR + i) * DST + col] = acc[i][j];
            }
        __syncthreads();
        // one thread per query row: stream the tile through the row's heap
        if (tid < ROWS && qbase + tid < n) {
            uint64_t* h = heap + tid;
            const int cols = static_cast<int>(min(static_cast<int64_t>(kTM), r_end - tbase));
            for (int col = 0; col < cols; ++col) {
                const uint64_t key = make_key(Dt[tid * DST + col],
                                              static_cast<uint32_t>(tbase + col));
                if (key < top) {
                    heap_replace_top<ROWS>(h, c, key);
                    top = h[0];
                }
            }
        }
    }
    __syncthreads();
    const int64_t S_ = cand.S;
    for (int e = tid; e < c * ROWS; e += kThreads) {
        const int row = e % ROWS, slot = e / ROWS;
        const int64_t q = qbase + row;
        if (q < n) cand.keys[(q * S_ + split) * c + slot] = heap[slot * ROWS + row];
    }
}

template <int METRIC, int ROWS>
cudaError_t launch_rows(const float* Q, int64_t n, const float* R, int64_t m, int32_t d,
                        const CandidateSet& cand, cudaStream_t st) {
    auto kern = cc_select_kernel<METRIC, ROWS>;
    const size_t smem = cc_smem_bytes<ROWS>(cand.c);
    cudaError_t err = allow_smem<cc_select_kernel<METRIC, ROWS>>(smem);
    if (err != cudaSuccess) return err;
    dim3 grid(static_cast<unsigned>((n + ROWS - 1) / ROWS), static_cast<unsigned>(cand.S));
    kern<<<grid, kThreads, smem, st>>>(Q, n, R, m, d, cand);
    return cudaGetLastError();
}

constexpr size_t kSmemCap = 220 * 1024;

}  // namespace

int cc_max_candidates() {
    int c = 16;
    while (cc_smem_bytes<16>(c + 16) <= kSmemCap) c += 16;
    return c;
}

cudaError_t launch_cc_select(const float* Q, int64_t n, const float* R, int64_t m, int32_t d,
                             int32_t metric, const CandidateSet& cand, cudaStream_t st,
                             int* launches) {
    const bool wide = cc_smem_bytes<64>(cand.c) <= kSmemCap;
    if (!wide && cc_smem_bytes<16>(cand.c) > kSmemCap) return cudaErrorInvalidValue;
    if (launches) ++*launches;
    if (metric == kL2)
        return wide ? launch_rows<kL2, 64>(Q, n, R, m, d, cand, st)
                    : launch_rows<kL2, 16>(Q, n, R, m, d, cand, st);
    if (metric == kL1)
        return wide ? launch_rows<kL1, 64>(Q, n, R, m, d, cand, st)
                    : launch_rows<kL1, 16>(Q, n, R, m, d, cand, st);
    return wide ? launch_rows<kLinf, 64>(Q, n, R, m, d, cand, st)
                : launch_rows<kLinf, 16>(Q, n, R, m, d, cand, st);
}

}  // namespace knn
