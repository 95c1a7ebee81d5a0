// knn_finalize.cu -- host side of the finalize and exact-fallback stages
// (launch shapes, launchers) and the self-join row pass.  The device code, and
// the description of the stages, is in finalize_device.cuh.
#include "finalize_device.cuh"

namespace knn {

// Self-join: row i of the (k+1)-neighbour result without reference i (or
// without its last entry when i is not among them).  One thread per row.
__global__ void drop_self_kernel(const float* __restrict__ din, const int32_t* __restrict__ iin,
                                 int64_t n, int32_t k, float* __restrict__ dout,
                                 int32_t* __restrict__ iout) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* dr = din + i * (k + 1);
    const int32_t* ir = iin + i * (k + 1);
    int o = 0;
    for (int s = 0; s <= k && o < k; ++s) {
        if (ir[s] == static_cast<int32_t>(i)) continue;
        dout[i * k + o] = dr[s];
        iout[i * k + o] = ir[s];
        ++o;
    }
}

cudaError_t launch_drop_self(const float* din, const int32_t* iin, int64_t n, int32_t k, float* dout,
                             int32_t* iout, cudaStream_t st, int* launches) {
    const unsigned grid = static_cast<unsigned>((n + 255) / 256);
    if (launches) ++*launches;
    drop_self_kernel<<<grid, 256, 0, st>>>(din, iin, n, k, dout, iout);
    return cudaGetLastError();
}

int finalize_max_pool() { return kMaxPool; }

template <int METRIC, int NV>
cudaError_t launch_finalize_nv(const FinalizeArgs& a, int P, int wpb, int se, size_t smem,
                               unsigned grid, cudaStream_t st) {
    cudaError_t err = allow_smem<finalize_kernel<METRIC, NV>>(smem);
    if (err != cudaSuccess) return err;
    finalize_kernel<METRIC, NV><<<grid, wpb * 32, smem, st>>>(a, P, wpb, se);
    return cudaGetLastError();
}

template <int METRIC>
cudaError_t launch_finalize_m(const FinalizeArgs& a, int nv, int P, int wpb, int se, size_t smem,
                              unsigned grid, cudaStream_t st) {
    switch (nv) {
        case 1: return launch_finalize_nv<METRIC, 1>(a, P, wpb, se, smem, grid, st);
        case 2: return launch_finalize_nv<METRIC, 2>(a, P, wpb, se, smem, grid, st);
        case 3: return launch_finalize_nv<METRIC, 3>(a, P, wpb, se, smem, grid, st);
        case 4: return launch_finalize_nv<METRIC, 4>(a, P, wpb, se, smem, grid, st);
        default: return launch_finalize_nv<METRIC, 0>(a, P, wpb, se, smem, grid, st);
    }
}

cudaError_t launch_finalize(const FinalizeArgs& a_in, cudaStream_t st, int* launches) {
    FinalizeArgs a = a_in;
    a.rel = f32_rel_bound(a.d);
    a.relf = static_cast<float>(2.02 * a.rel);
    a.ffw = static_cast<float>(2.5 * ff_rel_bound(a.d));
    int P = a.use_hits ? 2 * a.hits.c + 32 : a.cand.S * a.cand.c;
    P = (P + 3) & ~3;
    if (P > kMaxPool) return cudaErrorInvalidValue;
    // hit-list staging: kStage entries; when the queries do not fill the GPU
    // anyway, room for every list entry a query can have (up to 12288), so
    // long lists are still read from shared memory
    int se = a.use_hits ? kStage : 0;
    if (a.use_hits && a.n <= 256) {
        const int64_t all = static_cast<int64_t>(a.hits.S) * a.hits.cap;
        se = static_cast<int>(all < kStage ? kStage : (all > 12288 ? 12288 : all));
    }
    const size_t per_warp = warp_scratch_bytes(P, prefix_cap(P, a.k), a.use_hits ? 1 : a.cand.S,
                                               a.d, se);
    // up to eight warps per block and four blocks per SM when the scratch allows
    int wpb = static_cast<int>((52 * 1024) / per_warp);
    if (wpb < 8) wpb = static_cast<int>((96 * 1024) / per_warp);
    wpb = wpb < 1 ? 1 : (wpb > kFinThreads / 32 ? kFinThreads / 32 : wpb);
    const size_t smem = per_warp * wpb;
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    const unsigned grid = static_cast<unsigned>((a.n + wpb - 1) / wpb);
    // float4 rows need d % 4 == 0 and 16-byte aligned reference and query arrays
    const bool aligned =
        ((reinterpret_cast<uintptr_t>(a.R) | reinterpret_cast<uintptr_t>(a.Q)) & 15) == 0;
    const int nv = (aligned && (a.d & 3) == 0 && a.d <= 128) ? (a.d + 31) / 32 : 0;
    if (launches) ++*launches;
    if (a.metric == kL2) return launch_finalize_m<kL2>(a, nv, P, wpb, se, smem, grid, st);
    if (a.metric == kL1) return launch_finalize_m<kL1>(a, nv, P, wpb, se, smem, grid, st);
    return launch_finalize_m<kLinf>(a, nv, P, wpb, se, smem, grid, st);
}

template <int METRIC>
cudaError_t launch_fallback_m(const FinalizeArgs& a, double* scratch, int32_t slots, int32_t* done,
                              size_t smem, cudaStream_t st) {
    cudaError_t err = allow_smem<fallback_kernel<METRIC>>(smem);
    if (err != cudaSuccess) return err;
    // half of the scratch slots for spread queries, half for the rest (a lone
    // slot serves every queued query with one CTA)
    const int32_t spread = slots >= 2 ? slots / 2 : 0;
    const unsigned chunks = spread > 0 ? static_cast<unsigned>((a.m + kFbChunk - 1) / kFbChunk) : 1u;
    fallback_kernel<METRIC><<<dim3(chunks, static_cast<unsigned>(slots)), kFbThreads, smem, st>>>(
        a, scratch, done, spread);
    return cudaGetLastError();
}

cudaError_t launch_fallback(const FinalizeArgs& a, double* scratch, int32_t slots, int32_t* done,
                            cudaStream_t st, int* launches) {
    if (a.k > kFbMaxK) return cudaErrorInvalidValue;
    const size_t smem = static_cast<size_t>(kFbCand) * (sizeof(uint64_t) + sizeof(uint32_t)) +
                        (static_cast<size_t>(a.d) + 4) * sizeof(float);
    if (smem + sizeof(FbShared<kFbThreads>) + 16 > 227 * 1024) return cudaErrorInvalidValue;
    if (launches) ++*launches;
    if (a.metric == kL2) return launch_fallback_m<kL2>(a, scratch, slots, done, smem, st);
    if (a.metric == kL1) return launch_fallback_m<kL1>(a, scratch, slots, done, smem, st);
    return launch_fallback_m<kLinf>(a, scratch, slots, done, smem, st);
}

}  // namespace knn
