// knn_tc.cu -- tensor-core (tcgen05 / TMEM / TMA) stages of the Euclidean
// search: host side (tensor maps, the launch plan, launchers).  The device
// code, and the description of the method, is in tc_device.cuh.
#include "tc_device.cuh"

namespace knn {
using namespace ptx;
namespace {

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &qr) == cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

}  // namespace

// rows x kp operand seen as 3-D: (128 bytes of K) x rows x K blocks, so one box
// brings box_rows rows with all their K blocks, laid out block-major
// ([K block][row][128 bytes], 128-byte swizzle) as the MMA descriptors expect.
// Rows outside the tensor read as zero.
bool tc_make_map(CUtensorMap* map, const void* base, int64_t rows, int kp, int prec, int box_rows,
                 int box_kb) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const int elt = (prec == kBF16) ? 2 : 4;
    const int kb = kp * elt / kAtomBytes;
    cuuint64_t dims[3] = {static_cast<cuuint64_t>(kAtomBytes / elt), static_cast<cuuint64_t>(rows),
                          static_cast<cuuint64_t>(kb)};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(kp) * elt, static_cast<cuuint64_t>(kAtomBytes)};
    cuuint32_t box[3] = {static_cast<cuuint32_t>(kAtomBytes / elt), static_cast<cuuint32_t>(box_rows),
                         static_cast<cuuint32_t>(box_kb > 0 ? box_kb : kb)};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map,
                    prec == kBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                    3, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

namespace {

template <int PREC, bool PILOT, int KBT, int EPI = 0>
cudaError_t launch_kernel(const TcPlan& p, const CUtensorMap& mq, const CUtensorMap& mr,
                          const TcArgs& a, cudaStream_t st) {
    auto kern = tc_kernel<PREC, PILOT, KBT, EPI>;
    const size_t smem = tc_smem_bytes(p.kb, p.kbs, p.stages, PILOT, EPI != 0);
    cudaError_t err = allow_smem<tc_kernel<PREC, PILOT, KBT, EPI>>(smem);
    if (err != cudaSuccess) return err;
    dim3 grid(static_cast<unsigned>((a.n + kBlockM - 1) / kBlockM), static_cast<unsigned>(a.S));
    kern<<<grid, kTcThreads, smem, st>>>(mq, mr, a);
    return cudaGetLastError();
}

template <int PREC, bool PILOT>
cudaError_t dispatch_kb(const TcPlan& p, const CUtensorMap& mq, const CUtensorMap& mr,
                        const TcArgs& a, cudaStream_t st) {
    if (p.kbs == p.kb) {   // whole-tile stages: unrolled issue for the common row lengths
        if constexpr (!PILOT) {
            if (p.raw && p.pilot) {
                switch (p.kb) {
                    case 1: return launch_kernel<PREC, false, 1, 1>(p, mq, mr, a, st);
                    case 2: return launch_kernel<PREC, false, 2, 1>(p, mq, mr, a, st);
                    default: break;
                }
            }
            if (p.raw) {   // every reference appended
                switch (p.kb) {
                    case 1: return launch_kernel<PREC, false, 1, 2>(p, mq, mr, a, st);
                    case 2: return launch_kernel<PREC, false, 2, 2>(p, mq, mr, a, st);
                    default: break;
                }
            }
        }
        switch (p.kb) {
            case 1: return launch_kernel<PREC, PILOT, 1>(p, mq, mr, a, st);
            case 2: return launch_kernel<PREC, PILOT, 2>(p, mq, mr, a, st);
            default: break;
        }
    }
    if constexpr (!PILOT) {
        if (p.raw && p.pilot) return launch_kernel<PREC, false, 0, 1>(p, mq, mr, a, st);
        if (p.raw) return launch_kernel<PREC, false, 0, 2>(p, mq, mr, a, st);   // every reference
    }
    return launch_kernel<PREC, PILOT, 0>(p, mq, mr, a, st);
}

template <bool PILOT>
cudaError_t dispatch(const TcPlan& p, int prec, const CUtensorMap& mq, const CUtensorMap& mr,
                     const TcArgs& a, cudaStream_t st) {
    if (prec == kBF16) return dispatch_kb<kBF16, PILOT>(p, mq, mr, a, st);
    return dispatch_kb<kTF32, PILOT>(p, mq, mr, a, st);
}

TcArgs base_args(const TcPlan& p, int64_t n, int64_t m, int32_t* error_flag) {
    TcArgs a{};
    a.n = n;
    a.m = m;
    a.kb = p.kb;
    a.ksteps = p.ksteps;
    a.kbs = p.kbs;
    a.stages = p.stages;
    a.chunk = p.chunk;
    a.S = p.S;
    a.stride = p.stride;
    a.spt = p.spt;
    a.G = p.G;
    a.gps = 32 / p.gsize;
    a.cap = p.cap;
    a.append_all = p.pilot ? 0 : 1;
    a.error_flag = error_flag;
    return a;
}

}  // namespace

// Self-test of the bounded waits: one thread waits, with the given limit, on
// an mbarrier nothing arrives at; when the wait gives up it raises the error
// flag, as the search kernels do, and the kernel returns.
__global__ void wait_probe_kernel(int32_t* error_flag, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(&bar, 0, nullptr, limit_ns)) atomicExch(error_flag, 1);
}

cudaError_t launch_wait_probe(int32_t* error_flag, uint64_t limit_ns, cudaStream_t st) {
    wait_probe_kernel<<<1, 32, 0, st>>>(error_flag, limit_ns);
    return cudaGetLastError();
}

int tc_padded_dim(int32_t d, int prec) {
    const int step = (prec == kBF16) ? 64 : 32;   // whole 128-byte K blocks per row
    return (d + kAugCols + step - 1) / step * step;
}

TcPlan tc_plan(int64_t n, int64_t m, int32_t d, int32_t kp, int prec, int32_t c, int num_sms,
               size_t smem_limit, int64_t force_chunk) {
    const size_t kSmemLimit = smem_limit;
    TcPlan p{};
    const int elt = (prec == kBF16) ? 2 : 4;
    const int kstep = 32 / elt;                    // elements per MMA K step
    p.mt = 1;
    p.rb = kTileN;
    p.groups = kGroups;
    p.kb = kp * elt / kAtomBytes;
    p.ksteps = (d + kAugCols + kstep - 1) / kstep;
    p.stages = 0;
    // whole-tile stages (one TMA box and one wait per tile) when two fit,
    // else single-K-block stages, as many as fit
    // (raw hit staging with them when it also fits: rows of up to 2 K blocks)
    for (int s = 4; s >= 2 && p.stages == 0; --s)
        if (tc_smem_bytes(p.kb, p.kb, s, false) <= kSmemLimit) {
            p.kbs = p.kb;
            p.stages = s;
            p.raw = (p.kb <= 2 && tc_smem_bytes(p.kb, p.kb, s, false, true) <= kSmemLimit) ? 1 : 0;
        }
    if (p.stages == 0) {
        // one K block per stage; raw hit staging when it leaves at least three
        // stages (or as many as the codes would)
        int s_codes = 0, s_raw = 0;
        for (int s = kMaxStages; s >= 2 && s_codes == 0; --s)
            if (tc_smem_bytes(p.kb, 1, s, false) <= kSmemLimit) s_codes = s;
        for (int s = kMaxStages; s >= 2 && s_raw == 0; --s)
            if (tc_smem_bytes(p.kb, 1, s, false, true) <= kSmemLimit) s_raw = s;
        if (s_codes > 0) {
            p.kbs = 1;
            p.raw = (s_raw >= 3 || (s_raw > 0 && s_raw == s_codes)) ? 1 : 0;
            p.stages = p.raw ? s_raw : s_codes;
        }
    }
    if (p.stages == 0) return p;   // operand rows too long for shared memory
    const int64_t qtiles = (n + kBlockM - 1) / kBlockM;
    // reference splits: the fewest whose CTAs fill at least 85% of the last wave
    int64_t max_s = m / (4 * kTileN);
    if (max_s < 1) max_s = 1;
    if (max_s > 256) max_s = 256;
    int S = 1;
    double best = 0.0;
    for (int s = 1; s <= max_s; ++s) {
        const int64_t ctas = qtiles * s;
        const int64_t waves = (ctas + num_sms - 1) / num_sms;
        const double eff = static_cast<double>(ctas) / (static_cast<double>(waves) * num_sms);
        if (eff > best + 1e-9) { best = eff; S = s; }
        if (eff >= 0.85) break;
    }
    if (force_chunk > 0) {   // a given split length (whole tiles) instead of the wave fill
        const int64_t fc = (force_chunk + kTileN - 1) / kTileN * kTileN;
        S = static_cast<int>((m + fc - 1) / fc);
    }
    int64_t chunk = (m + S - 1) / S;
    chunk = (chunk + kTileN - 1) / kTileN * kTileN;
    S = static_cast<int>((m + chunk - 1) / chunk);
    p.S = S;
    p.chunk = chunk;
    // pilot sampling: every stride-th tile (one reference in 16 or fewer), at
    // most ~1024 groups of 32 per query
    int gpt = kTileN / 32;                         // groups per tile
    p.gsize = 32;
    const int64_t tiles_total = (m + kTileN - 1) / kTileN;
    int stride = 4096 / kTileN;
    while (tiles_total * gpt / stride > 1024) stride *= 2;
    const int tps = static_cast<int>(chunk / kTileN);
    // c' = lambda + 4 sqrt(lambda) + 4, lambda = the expected number of
    // sampled references among the c best (c times the sampled fraction: each
    // split samples its tiles 0, stride, 2 stride, ..., so a short split
    // samples a larger share).  At least c' sampled references pass the
    // threshold; were fewer than c to pass overall, all would be among the c
    // best, so at least c' of the c best were sampled: a Poisson(lambda) tail,
    // about 4e-6 per query at lambda = 5.3, c' = 19 (n = m = 38400, k = 20).
    // Such a query is finished by the exact fallback.  The c'-th largest of G
    // group maxima needs G comfortably above c': sample denser (halve the
    // stride) until G >= c' + 8, and run no pilot (every reference appended)
    // only when even every tile does not give that many groups.
    // When every tile is sampled the count is no longer a random draw: c' = c
    // groups reaching T put at least c references above it.  Should even that
    // leave too few groups of 32, the groups shrink to 16 or 8 references
    // (the elements u = i mod 2 or mod 4 of a 32-column slice, group i).
    // The group slots of a short split's missing tiles, and groups past the
    // end of the data, hold no maximum: gvalid counts the real groups.
    int64_t gvalid = 0;
    for (;;) {
        p.stride = stride;
        p.spt = (tps + stride - 1) / stride;
        p.G = S * p.spt * gpt;
        const int gps = 32 / p.gsize;
        int64_t sampled = 0;
        gvalid = 0;
        for (int s = 0; s < S; ++s) {
            const int64_t rows = std::min<int64_t>(m - s * chunk, chunk);
            const int64_t tiles = (rows + kTileN - 1) / kTileN;
            for (int64_t t = 0; t < tiles; t += stride) {
                const int64_t v = std::min<int64_t>(rows - t * kTileN, kTileN);
                sampled += v;
                // slice j of the tile holds min(32, v - 32 j) elements, of
                // which its first gps each start a group
                for (int64_t j = 0; j * 32 < v; ++j) gvalid += std::min<int64_t>(v - 32 * j, gps);
            }
        }
        const double lambda = static_cast<double>(c) * static_cast<double>(sampled) / static_cast<double>(m);
        p.cprime = sampled == m ? c
                                : static_cast<int>(std::ceil(lambda + 4.0 * std::sqrt(lambda) + 4.0));
        if (gvalid >= p.cprime + 8 || p.G > 1024) break;
        if (stride > 1) {
            stride /= 2;
        } else if (p.gsize > 8) {
            p.gsize /= 2;
            gpt *= 2;
        } else {
            break;
        }
    }
    // the threshold kernel holds at most 64 x 32 group maxima per query
    p.pilot = (gvalid >= p.cprime + 8 && p.G <= 2048) ? 1 : 0;
    // list capacity per (query, split, column group).  The threshold is the
    // c'-th largest of gvalid group maxima (groups of gsize): a fraction
    // pg = c'/gvalid of the groups reach it, so about f = 1 - (1 - pg)^(1/gsize)
    // of all references pass, m f in all.  That count varies from query to
    // query with the order statistic (about 1/sqrt(c') relative) and its
    // split over the lists: 2.5 times the mean per list plus 48 keeps
    // overflows (sent to the exact fallback) rare.
    if (p.pilot) {
        const double pg = std::min(1.0, static_cast<double>(p.cprime) / static_cast<double>(gvalid));
        const double f = 1.0 - std::pow(1.0 - pg, 1.0 / static_cast<double>(p.gsize));
        const double per_list = static_cast<double>(m) * f / (kGroups * S);
        int64_t cap = static_cast<int64_t>(std::ceil(2.5 * per_list)) + 48;
        if (cap > chunk / kGroups) cap = chunk / kGroups;
        p.cap = static_cast<int32_t>((cap + 31) / 32 * 32);
    } else {
        p.cap = static_cast<int32_t>(chunk / kGroups);
    }
    p.smem_filter = tc_smem_bytes(p.kb, p.kbs, p.stages, false, p.raw != 0);
    return p;
}

cudaError_t launch_prepare_ref(const float* R, int64_t m, int32_t d, int32_t kp, int prec,
                               void* R_lp, float* norms, uint32_t* rmax2, cudaStream_t st,
                               int* launches) {
    cudaError_t err = cudaMemsetAsync(rmax2, 0, sizeof(uint32_t), st);
    if (err != cudaSuccess) return err;
    const int64_t warps = (m + kPrepRowsPerWarp - 1) / kPrepRowsPerWarp;
    const unsigned grid = static_cast<unsigned>((warps * 32 + 255) / 256);
    if (prec == kBF16)
        prepare_kernel<kBF16, true><<<grid, 256, 0, st>>>(R, m, d, kp, R_lp, norms, rmax2, nullptr,
                                                           nullptr);
    else
        prepare_kernel<kTF32, true><<<grid, 256, 0, st>>>(R, m, d, kp, R_lp, norms, rmax2, nullptr,
                                                           nullptr);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_prepare_query(const float* Q, int64_t n, int32_t d, int32_t kp, int prec,
                                 void* Q_lp, const HitScale& qs, float* Q_copy, cudaStream_t st,
                                 int* launches) {
    const int64_t warps = (n + kPrepRowsPerWarp - 1) / kPrepRowsPerWarp;
    const unsigned grid = static_cast<unsigned>((warps * 32 + 255) / 256);
    if (prec == kBF16)
        prepare_kernel<kBF16, false><<<grid, 256, 0, st>>>(Q, n, d, kp, Q_lp, nullptr,
                                                            const_cast<uint32_t*>(qs.rmax2), qs.qscale,
                                                            Q_copy);
    else
        prepare_kernel<kTF32, false><<<grid, 256, 0, st>>>(Q, n, d, kp, Q_lp, nullptr,
                                                            const_cast<uint32_t*>(qs.rmax2), qs.qscale,
                                                            Q_copy);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_tc_pilot(const TcPlan& p, const void* Q_lp, int64_t n, const void* R_lp, int64_t m,
                            int32_t kp, int prec, uint32_t* gmax, int32_t* error_flag, cudaStream_t st,
                            int* launches) {
    CUtensorMap mq, mr;
    if (!tc_make_map(&mq, Q_lp, n, kp, prec, kBlockM, 0) || !tc_make_map(&mr, R_lp, m, kp, prec, p.rb, p.kbs))
        return cudaErrorInvalidValue;
    TcArgs a = base_args(p, n, m, error_flag);
    a.gmax = gmax;   // every slot of every row is written by the pilot
    if (launches) ++*launches;
    return dispatch<true>(p, prec, mq, mr, a, st);
}

template <int PREC, int VPL>
void launch_threshold_vpl(const TcPlan& p, const uint32_t* gmax, int64_t n, int32_t d, int32_t kp,
                          void* Q_lp, const HitScale& qs, cudaStream_t st) {
    constexpr int wpb = 8;
    const unsigned grid = static_cast<unsigned>((n + wpb - 1) / wpb);
    threshold_kernel<PREC, VPL><<<grid, wpb * 32, 0, st>>>(gmax, n, p.G, p.cprime, d, kp, Q_lp,
                                                          qs.rmax2, qs.qscale);
}

template <int PREC>
cudaError_t launch_threshold_p(const TcPlan& p, const uint32_t* gmax, int64_t n, int32_t d,
                               int32_t kp, void* Q_lp, const HitScale& qs, cudaStream_t st) {
    const int vpl = (p.G + 31) / 32;
    if (vpl <= 1) launch_threshold_vpl<PREC, 1>(p, gmax, n, d, kp, Q_lp, qs, st);
    else if (vpl <= 2) launch_threshold_vpl<PREC, 2>(p, gmax, n, d, kp, Q_lp, qs, st);
    else if (vpl <= 4) launch_threshold_vpl<PREC, 4>(p, gmax, n, d, kp, Q_lp, qs, st);
    else if (vpl <= 8) launch_threshold_vpl<PREC, 8>(p, gmax, n, d, kp, Q_lp, qs, st);
    else if (vpl <= 16) launch_threshold_vpl<PREC, 16>(p, gmax, n, d, kp, Q_lp, qs, st);
    else if (vpl <= 32) launch_threshold_vpl<PREC, 32>(p, gmax, n, d, kp, Q_lp, qs, st);
    else if (vpl <= 64) launch_threshold_vpl<PREC, 64>(p, gmax, n, d, kp, Q_lp, qs, st);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_tc_threshold(const TcPlan& p, const uint32_t* gmax, int64_t n, int32_t d,
                                int32_t kp, int prec, void* Q_lp, const HitScale& qs,
                                cudaStream_t st, int* launches) {
    if (launches) ++*launches;
    if (prec == kBF16) return launch_threshold_p<kBF16>(p, gmax, n, d, kp, Q_lp, qs, st);
    return launch_threshold_p<kTF32>(p, gmax, n, d, kp, Q_lp, qs, st);
}

cudaError_t launch_tc_filter(const TcPlan& p, const void* Q_lp, int64_t n, const void* R_lp, int64_t m,
                             int32_t kp, int prec, uint64_t* lists, int32_t* counts,
                             const float* qscale, int32_t* error_flag, cudaStream_t st,
                             int* launches) {
    CUtensorMap mq, mr;
    if (!tc_make_map(&mq, Q_lp, n, kp, prec, kBlockM, 0) || !tc_make_map(&mr, R_lp, m, kp, prec, p.rb, p.kbs))
        return cudaErrorInvalidValue;
    TcArgs a = base_args(p, n, m, error_flag);
    a.stride = 1;
    a.lists = lists;
    a.counts = counts;
    a.qscale = qscale;
    if (launches) ++*launches;
    return dispatch<false>(p, prec, mq, mr, a, st);
}

}  // namespace knn
