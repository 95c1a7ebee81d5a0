// knn_small.cu -- float32 select for small reference sets: every distance of
// a query held in shared memory and the c smallest found by an exact
// selection, with no data-dependent serial work.
//
// Steps 1-3 of the brute-force algorithm of Sec. 2.1 for one query per warp:
// the CTA's eight warps share reference tiles staged in shared memory
// (asynchronous copies, the next tile in flight while one is used), each
// lane computes the float32 distances of its references (coordinate
// differences, coordinate 0 first, as the other float32 stages do) into the
// warp's row of m distances; then the c-th smallest distance is found by a
// bisection over the order-preserving bit patterns (each step a warp-wide
// count), and the keys below it, plus the lowest-index ones equal to it, are
// compacted in index order by ballots.  The output is a candidate set with one
// split per query of at least the c nearest keys (a few spare slots let the
// bisection stop at the first midpoint whose count fits them; unused slots
// are empty), the finalize's float32 input.
//
// For reference sets of a few thousand points the heap-based select spends
// its time in the first tiles, where almost every distance enters the heap
// one after another in divergent code; here every step is the same for all
// lanes.
#include "knn_internal.cuh"

namespace knn {
namespace {

constexpr int kWarps = 8;                 // queries per CTA
constexpr int kThreads = 32 * kWarps;
constexpr int kTileFloats = 6144;         // one staged reference tile (24 KB), two in flight

// Row pitch (floats) of a staged reference or query: d rounded up to whole
// float4s, plus one more float4 when that count is even, so that the 16-byte
// loads of a quarter warp (eight rows an odd number of float4s apart) fall on
// distinct banks.
__host__ __device__ inline int small_pitch(int32_t d) {
    int v = (d + 3) / 4;
    if ((v & 1) == 0) ++v;
    return 4 * v;
}
// References per staged tile: as many whole warps' worth (multiples of 32) as
// fill kTileFloats, at least 32.
__host__ __device__ inline int small_tile_rows(int32_t d) {
    const int r = kTileFloats / small_pitch(d) / 32 * 32;
    return r < 32 ? 32 : r;
}

// Asynchronous copies global -> shared of 4 or 16 bytes; src_bytes 0 writes zeros.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int METRIC>
__device__ __forceinline__ float term(float acc, float diff) {
    if (METRIC == kL2) return fmaf(diff, diff, acc);
    if (METRIC == kL1) return acc + fabsf(diff);
    return fmaxf(acc, fabsf(diff));
}

// PER: distances per lane held in registers for the selection (m <= 32 PER).
// c_need: the fewest keys a query keeps (its c nearest); cand.c >= c_need
// slots, the spare ones let the bisection stop early.
template <int METRIC, int PER>
__global__ void __launch_bounds__(kThreads)
small_select_kernel(const float* __restrict__ Q, int64_t n, const float* __restrict__ R,
                    int32_t m, int32_t d, int32_t c_need, CandidateSet cand) {
    extern __shared__ __align__(16) float sm[];
    const int p = small_pitch(d);
    const int TR = small_tile_rows(d);
    float* Rt = sm;                         // [2][TR][p], double buffered
    float* Qw = Rt + 2 * TR * p;            // [kWarps][p]
    float* Dw = Qw + kWarps * p;            // [kWarps][m]
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t q = static_cast<int64_t>(blockIdx.x) * kWarps + warp;
    const bool live = q < n;
    float* qrow = Qw + warp * p;
    float* drow = Dw + static_cast<size_t>(warp) * m;
    for (int t = lane; t < p; t += 32) qrow[t] = (live && t < d) ? Q[q * d + t] : 0.f;
    const int nv = p / 4;
    const int ntiles = (m + TR - 1) / TR;
    // tile b -> buffer b & 1: every thread issues its copies (zero beyond the
    // rows and coordinates) without waiting for any of them; the tile is walked
    // as one flat sequence of 16-byte units (rows of d % 4 == 0 floats, 16-byte
    // aligned in global memory) or of floats, thread i taking units i, i + 256,
    // ..., its (row, unit) position advanced incrementally
    const bool vec = (d & 3) == 0 && (reinterpret_cast<uintptr_t>(R) & 15) == 0;
    const int upr = vec ? p / 4 : p;                  // units per staged row
    const int dun = vec ? d / 4 : d;                  // units holding data
    const int step_r = kThreads / upr, step_u = kThreads % upr;
    auto stage = [&](int b) {
        float* dst = Rt + (b & 1) * TR * p;
        const int base = b * TR;
        const int rows = min(TR, m - base);
        int r = threadIdx.x / upr, u = threadIdx.x % upr;
        while (r < TR) {
            const bool ok = r < rows && u < dun;
            const float* src = ok ? R + static_cast<int64_t>(base + r) * d + (vec ? 4 * u : u) : R;
            if (vec) cp_async16(dst + r * p + 4 * u, src, ok ? 16 : 0);
            else cp_async4(dst + r * p + u, src, ok ? 4 : 0);
            r += step_r;
            u += step_u;
            if (u >= upr) {
                u -= upr;
                ++r;
            }
        }
        cp_async_commit();
    };
    stage(0);
    for (int b = 0; b < ntiles; ++b) {
        if (b + 1 < ntiles) {
            stage(b + 1);
            cp_async_wait<1>();    // this thread's copies of tile b have landed
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();           // everyone's have (and the query rows are staged)
        const int base = b * TR;
        const int rows = min(TR, m - base);
        const float* Rb = Rt + (b & 1) * TR * p;
        const float4* q4 = reinterpret_cast<const float4*>(qrow);
        for (int rr = lane; rr < rows; rr += 32) {
            const float4* r4 = reinterpret_cast<const float4*>(Rb + rr * p);
            float acc = 0.f;
            for (int v = 0; v < nv; ++v) {
                const float4 x = r4[v], y = q4[v];
                acc = term<METRIC>(acc, y.x - x.x);
                acc = term<METRIC>(acc, y.y - x.y);
                acc = term<METRIC>(acc, y.z - x.z);
                acc = term<METRIC>(acc, y.w - x.w);
            }
            drow[base + rr] = acc;
        }
        __syncthreads();           // buffer b & 1 is free for tile b + 2
    }
    __syncwarp();
    if (!live) return;   // no block-wide barrier follows

    // distances are >= 0: their bit patterns order like the values; the
    // lane's (j = lane + 32 i) go to registers, absent ones as all-ones, which
    // no count below reaches
    const unsigned full = 0xffffffffu;
    uint32_t v[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int j = lane + 32 * i;
        v[i] = j < m ? __float_as_uint(drow[j]) : 0xffffffffu;
    }
    uint32_t lo = 0xffffffffu, hi = 0u;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        lo = min(lo, v[i]);
        if (lane + 32 * i < m) hi = max(hi, v[i]);
    }
    lo = __reduce_min_sync(full, lo);
    hi = __reduce_max_sync(full, hi);
    const int slots = cand.c;
    // tau: a pattern with c_need <= count(<= tau), found by bisection from
    // [lo, hi] (count(<= hi) = m >= c_need); it stops at the first midpoint
    // whose count also fits the slots, else ends at the smallest such pattern
    uint32_t a = lo, b = hi;
    int cnt_b = m;
    while (a < b && cnt_b > slots) {
        const uint32_t mid = a + (b - a) / 2;
        int cnt = 0;
#pragma unroll
        for (int i = 0; i < PER; ++i) cnt += v[i] <= mid ? 1 : 0;
        cnt = static_cast<int>(__reduce_add_sync(full, static_cast<unsigned>(cnt)));
        if (cnt >= c_need) {
            b = mid;
            cnt_b = cnt;
        } else {
            a = mid + 1;
        }
    }
    const uint32_t tau = b;
    int below = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) below += v[i] < tau ? 1 : 0;
    below = static_cast<int>(__reduce_add_sync(full, static_cast<unsigned>(below)));
    // every key below tau, then keys equal to it, lowest indices first, up to
    // the slots: a key left out is never below one kept
    const int need_eq = min(cnt_b, slots) - below;
    uint64_t* out = cand.keys + (q * cand.S) * slots;
    const unsigned lt_mask = (1u << lane) - 1u;
    int pos = 0, eq_seen = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        if (32 * i >= m) break;
        const int j = lane + 32 * i;
        const uint32_t u = v[i];
        const bool eq = j < m && u == tau;
        const unsigned beq = __ballot_sync(full, eq);
        const bool take = (j < m && u < tau) || (eq && eq_seen + __popc(beq & lt_mask) < need_eq);
        const unsigned bt = __ballot_sync(full, take);
        if (take) out[pos + __popc(bt & lt_mask)] = make_key(__uint_as_float(u), static_cast<uint32_t>(j));
        pos += __popc(bt);
        eq_seen += __popc(beq);
    }
    for (int e = pos + lane; e < slots; e += 32) out[e] = kEmptyKey;
}

template <int METRIC, int PER>
cudaError_t launch_per(const float* Q, int64_t n, const float* R, int64_t m, int32_t d,
                       int32_t c_need, const CandidateSet& cand, size_t smem, cudaStream_t st) {
    cudaError_t err = allow_smem<small_select_kernel<METRIC, PER>>(smem);
    if (err != cudaSuccess) return err;
    const unsigned grid = static_cast<unsigned>((n + kWarps - 1) / kWarps);
    small_select_kernel<METRIC, PER><<<grid, kThreads, smem, st>>>(Q, n, R, static_cast<int32_t>(m),
                                                                   d, c_need, cand);
    return cudaGetLastError();
}

template <int METRIC>
cudaError_t launch_metric(const float* Q, int64_t n, const float* R, int64_t m, int32_t d,
                          int32_t c_need, const CandidateSet& cand, size_t smem, cudaStream_t st) {
    if (m <= 32 * 16) return launch_per<METRIC, 16>(Q, n, R, m, d, c_need, cand, smem, st);
    if (m <= 32 * 32) return launch_per<METRIC, 32>(Q, n, R, m, d, c_need, cand, smem, st);
    if (m <= 32 * 48) return launch_per<METRIC, 48>(Q, n, R, m, d, c_need, cand, smem, st);
    if (m <= 32 * 64) return launch_per<METRIC, 64>(Q, n, R, m, d, c_need, cand, smem, st);
    return launch_per<METRIC, 128>(Q, n, R, m, d, c_need, cand, smem, st);
}

}  // namespace

size_t small_select_smem(int64_t m, int32_t d) {
    const size_t p = static_cast<size_t>(small_pitch(d));
    const size_t tr = static_cast<size_t>(small_tile_rows(d));
    return sizeof(float) * (2 * tr * p + kWarps * p + kWarps * static_cast<size_t>(m));
}

bool small_select_fits(int64_t m, int32_t d) {
    return m >= 1 && m <= kSmallSelectMaxM && small_select_smem(m, d) <= 220 * 1024;
}

cudaError_t launch_small_select(const float* Q, int64_t n, const float* R, int64_t m, int32_t d,
                                int32_t metric, int32_t c_need, const CandidateSet& cand,
                                cudaStream_t st, int* launches) {
    if (!small_select_fits(m, d) || cand.S != 1 || c_need < 1 || c_need > m || cand.c < c_need)
        return cudaErrorInvalidValue;
    const size_t smem = small_select_smem(m, d);
    if (launches) ++*launches;
    if (metric == kL2) return launch_metric<kL2>(Q, n, R, m, d, c_need, cand, smem, st);
    if (metric == kL1) return launch_metric<kL1>(Q, n, R, m, d, c_need, cand, smem, st);
    return launch_metric<kLinf>(Q, n, R, m, d, c_need, cand, smem, st);
}

}  // namespace knn
