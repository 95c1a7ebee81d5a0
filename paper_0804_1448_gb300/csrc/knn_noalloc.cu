// knn_noalloc.cu -- the float32 search with a statically reserved scratch area
// and no allocation at all (knn_search_static in include/knn.h).
//
// Some callers cannot allocate device memory at the moment they search:
// frameworks that hand out every device allocation from their own pool (and
// account for it), and latency-bound paths that cannot afford the implicit
// device synchronisation of cudaMalloc/cudaFree.
// For them this file runs the same three stages as the float32 form of
// knn_search (fused distance + top-c select, finalize, exact fallback), with
// every intermediate placed in one file-scope __device__ array.
//
// The array is part of the library's device image: every GPU that loads the
// library holds its kStaticScratchBytes until the process exits.  In host code
// the array's name is only a host-side stand-in, so its device address is
// looked up with cudaGetSymbolAddress, once per device, with that device
// current, on the first call made on that device.
#include <cstring>
#include <mutex>

#include "../../include/knn.h"
#include "knn_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = 32ull << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct DeviceScratch {
    unsigned char* base = nullptr;   // device address of g_static_scratch on this device
    int num_sms = 0;
};
DeviceScratch g_devices[kMaxDevices];
std::mutex g_setup_mutex;

// Counters at the head of the scratch area (cleared by every call).
struct StaticCounters {
    int32_t fallback_count;
    int32_t pad;
    unsigned long long recheck_total;
    unsigned long long fallback_total;
    unsigned long long fallback_reason[4];
    int32_t fb_done[64];   // the fallback's chunk counters (zeroed with the rest)
};

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

knn_status device_scratch(int device, DeviceScratch* out) {
    if (device < 0 || device >= kMaxDevices) return KNN_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceScratch& ds = g_devices[device];
    if (!ds.base) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return KNN_ERR_CUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
            (void)cudaGetLastError();
            return KNN_ERR_CUDA;
        }
        ds.base = static_cast<unsigned char*>(p);
        ds.num_sms = sms;
    }
    *out = ds;
    return KNN_OK;
}

}  // namespace

using namespace knn;

extern "C" knn_status knn_search_static(const float* R, int64_t m, const float* Q, int64_t n,
                                        int32_t d, int32_t k, knn_metric metric, float* dist_out,
                                        int32_t* idx_out, void* cuda_stream) {
    if (m < 1 || n < 0 || d < 1 || k < 1 || k > m ||
        (metric != KNN_L2 && metric != KNN_L1 && metric != KNN_LINF))
        return KNN_ERR_INVALID;
    if (!R || (n > 0 && (!Q || !dist_out || !idx_out))) return KNN_ERR_INVALID;
    if (k > KNN_K_MAX || m > 0x7fffffffLL || n > 0x7fffffffLL) return KNN_ERR_UNSUPPORTED;
    if (n == 0) return KNN_OK;

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        (void)cudaGetLastError();
        return KNN_ERR_CUDA;
    }
    DeviceScratch ds;
    knn_status st = device_scratch(device, &ds);
    if (st != KNN_OK) return st;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

    // same candidate count and reference splits as the float32 form of knn_search
    const int margin = k / 4 > 8 ? k / 4 : 8;
    int c = k + margin;
    if (c > cc_max_candidates()) c = cc_max_candidates();
    if (c > m) c = static_cast<int>(m);
    if (c < k) return KNN_ERR_UNSUPPORTED;
    int64_t chunk = 0;
    const int S = cc_plan_splits(n, m, c, ds.num_sms, finalize_max_pool(), &chunk);
    if (static_cast<int64_t>(S) * c > finalize_max_pool()) return KNN_ERR_UNSUPPORTED;

    // layout of the static scratch: counters, candidates, fallback queue, and
    // whatever is left for the exact fallback (fb_grid x m doubles)
    const size_t off_ctr = 0;
    const size_t off_cand = align256(sizeof(StaticCounters));
    const size_t cand_bytes = static_cast<size_t>(n) * S * c * sizeof(uint64_t);
    const size_t off_list = align256(off_cand + cand_bytes);
    const size_t off_fb = align256(off_list + static_cast<size_t>(n) * sizeof(int32_t));
    if (off_fb + static_cast<size_t>(m) * sizeof(double) > kStaticScratchBytes)
        return KNN_ERR_UNSUPPORTED;   // the problem does not fit the static scratch
    int64_t fb_grid = static_cast<int64_t>((kStaticScratchBytes - off_fb) / (sizeof(double) * m));
    if (fb_grid > 64) fb_grid = 64;

    unsigned char* base = ds.base;
    StaticCounters* ctr = reinterpret_cast<StaticCounters*>(base + off_ctr);
    if (cudaMemsetAsync(ctr, 0, sizeof(StaticCounters), stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return KNN_ERR_CUDA;
    }
    CandidateSet cs;
    cs.keys = reinterpret_cast<uint64_t*>(base + off_cand);
    cs.n = n;
    cs.S = S;
    cs.c = c;
    cs.chunk = chunk;
    cs.exact = 1;
    int launches = 0;
    cudaError_t err = launch_cc_select(Q, n, R, m, d, metric, cs, stream, &launches);
    FinalizeArgs fa{};
    fa.use_hits = 0;
    fa.cand = cs;
    fa.Q = Q;
    fa.R = R;
    fa.n = n;
    fa.m = m;
    fa.d = d;
    fa.k = k;
    fa.metric = metric;
    fa.dist_out = dist_out;
    fa.idx_out = idx_out;
    fa.fallback_count = &ctr->fallback_count;
    fa.fallback_list = reinterpret_cast<int32_t*>(base + off_list);
    fa.recheck_counter = &ctr->recheck_total;
    fa.fallback_total = &ctr->fallback_total;
    fa.fallback_reason = ctr->fallback_reason;
    if (err == cudaSuccess) err = launch_finalize(fa, stream, &launches);
    if (err == cudaSuccess)
        err = launch_fallback(fa, reinterpret_cast<double*>(base + off_fb),
                              static_cast<int32_t>(fb_grid), ctr->fb_done, stream, &launches);
    if (err != cudaSuccess) {
        (void)cudaGetLastError();
        return KNN_ERR_CUDA;
    }
    return KNN_OK;
}
