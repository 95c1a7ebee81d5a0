// knn_tc.cu -- tensor-core (tcgen05 / TMEM / TMA) stages of the Euclidean search.
//
// For a fixed query q the Euclidean ranking of the references depends only on
// score(q, r) = ||r||^2 - 2 q.r  (||q - r||^2 = ||q||^2 + score).  The tensor
// cores compute an augmented product in one pass over K:
//     query row      [q_0 .. q_{d-1},  1,        1,        t_hi, t_lo, 0 ..]
//     reference row  [r_0 .. r_{d-1}, -nr_hi/2, -nr_lo/2,  1,    1,    0 ..]
//     acc = q.r - ||r||^2/2 + t = (2t - score) / 2
// where nr_hi + nr_lo is ||r||^2 split into two low-precision words, and
// t_hi + t_lo a per-query threshold t (0 in the pilot pass).  Larger acc is
// nearer.  Two passes use it:
//   pilot   -- on every stride-th reference tile, the maximum acc of each
//              group of 32 references (t = 0); a per-query order statistic of
//              these group maxima is a threshold that at least c' references
//              (sampled ones) pass, and about c'*stride references overall;
//   filter  -- on every tile, the sign bit of acc says whether the reference
//              passes the query's threshold (acc >= 0); passing references are
//              appended, with their acc, to the query's list.  A funnel shift
//              per element collects the sign bits, so the common case costs one
//              instruction per distance.
// The lists then go to the finalize stage (knn_finalize.cu), which keeps the
// best c by acc, re-ranks them with exact float32 differences, and checks the
// list was neither too short nor overflowed.
//
// CTA layout: MT tiles of 128 queries (MMA M; one TMEM lane per query) share
// every reference tile of 128 (MMA N):
//   warp 0        TMA producer: the query tiles once, then reference tiles into
//                 a ring of `stages` shared-memory buffers (128-byte swizzle);
//   warp 1        MMA issuer: per reference tile and query tile, kp*elt/32
//                 tcgen05.mma into one of two TMEM accumulators per query tile;
//                 tcgen05.commit frees the smem stage and publishes the tile;
//   warps 2..     epilogue, 4 per query tile: thread t of warp w owns the query
//                 row 32*(w%4)+t; tcgen05.ld 32x32b reads 32 columns at a time.
// Every mbarrier wait is bounded; on expiry the CTA raises the error flag,
// stops, waits for what it issued and frees its TMEM.
#include <cmath>

#include <cuda_bf16.h>

#include "knn_internal.cuh"
#include "tc_ptx.cuh"

namespace knn {
using namespace ptx;
namespace {

constexpr int kBlockM = 128;
constexpr int kBlockN = 128;
constexpr int kAtomBytes = 128;
constexpr int kTileBytes = kBlockM * kAtomBytes;   // one 128-byte K block of 128 rows
constexpr int kMaxStages = 12;
constexpr size_t kSmemLimit = 232448;
constexpr int kAugCols = 4;

struct TcArgs {
    int64_t n, m;
    int32_t kb, ksteps, stages;
    int64_t chunk;        // references per split (multiple of kBlockN)
    int32_t S;
    int32_t stride;       // pilot: every stride-th tile of a split
    int32_t spt;          // pilot: sampled-tile slots per split
    int32_t G;            // pilot: group maxima per query (S * spt * 4)
    uint32_t* gmax;       // pilot: [n][G] order-mapped maxima, 0 = no group
    uint64_t* lists;      // filter: [n][S][cap]
    int32_t* counts;      // filter: [n][S] (may exceed cap: overflow)
    int32_t cap;
    int32_t append_all;   // filter: every valid reference passes
    int32_t* error_flag;
};

// A: mt query tiles of kb K blocks (resident); B: a ring of `stages` single
// K blocks of one reference tile; staging of hit values (filter only).
__host__ __device__ constexpr size_t tc_smem_bytes(int mt, int kb, int stages, bool pilot) {
    return 1024 + static_cast<size_t>(kTileBytes) * (static_cast<size_t>(mt) * kb + stages) +
           (pilot ? 0 : static_cast<size_t>(128) * mt * 32 * 4) + 512;
}

template <int PREC, int MT, bool PILOT>
__global__ void __launch_bounds__(64 + 128 * MT, 1)
tc_kernel(const __grid_constant__ CUtensorMap tmap_q, const __grid_constant__ CUtensorMap tmap_r,
          TcArgs a) {
    constexpr int kEpi = 128 * MT;
    constexpr uint32_t kTmemCols = 256 * MT;   // two 128-column accumulators per query tile
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);

    const int KB = a.kb, NST = a.stages;
    unsigned char* sA = smem;
    unsigned char* sB = sA + static_cast<size_t>(MT) * KB * kTileBytes;
    float* stage = reinterpret_cast<float*>(sB + static_cast<size_t>(NST) * kTileBytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(stage + (PILOT ? 0 : kEpi * 32));
    uint64_t* full = bars;
    uint64_t* empty = bars + kMaxStages;
    uint64_t* a_full = bars + 2 * kMaxStages;
    uint64_t* t_full = a_full + 1;
    uint64_t* t_empty = t_full + 2;
    uint64_t* drain = t_empty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t q0 = static_cast<int64_t>(blockIdx.x) * kBlockM * MT;
    const int split = blockIdx.y;
    const int64_t r_begin = static_cast<int64_t>(split) * a.chunk;
    const int64_t r_end = min(a.m, r_begin + a.chunk);
    const int tiles_all = static_cast<int>((r_end - r_begin + kBlockN - 1) / kBlockN);
    const int stride = PILOT ? a.stride : 1;
    const int nt = (tiles_all + stride - 1) / stride;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(a_full, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&t_full[b], 1);
            mbar_init(&t_empty[b], kEpi);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    auto fail = [&]() {
        *abort_flag = 1;
        atomicExch(a.error_flag, 1);
    };

    if (warp == 0) {
        // -------------------------------------------------------- producer
        if (lane == 0) {
            constexpr int box_x = kAtomBytes / ((PREC == kBF16) ? 2 : 4);
            mbar_expect_tx(a_full, MT * KB * kTileBytes);
            for (int mt = 0; mt < MT; ++mt)
                for (int kb = 0; kb < KB; ++kb)
                    tma_load_2d(sA + static_cast<size_t>(mt * KB + kb) * kTileBytes, &tmap_q, a_full,
                                kb * box_x, static_cast<int>(q0 + mt * kBlockM));
            int issued = 0;   // K blocks issued; block g goes to stage g % NST
            bool ok = true;
            for (int i = 0; ok && i < nt; ++i) {
                const int y = static_cast<int>(r_begin + static_cast<int64_t>(i) * stride * kBlockN);
                for (int kb = 0; kb < KB; ++kb) {
                    const int g = i * KB + kb, s = g % NST;
                    if (!mbar_wait(&empty[s], ((g / NST) & 1) ^ 1, abort_flag)) { fail(); ok = false; break; }
                    mbar_expect_tx(&full[s], kTileBytes);
                    tma_load_2d(sB + static_cast<size_t>(s) * kTileBytes, &tmap_r, &full[s],
                                kb * box_x, y);
                    issued = g + 1;
                }
            }
            mbar_wait(a_full, 0, nullptr);   // drain: every issued copy has landed
            for (int g = (issued > NST ? issued - NST : 0); g < issued; ++g)
                mbar_wait(&full[g % NST], (g / NST) & 1, nullptr);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t id = idesc(PREC == kBF16 ? 1 : 2, kBlockM, kBlockN);
            bool ok = mbar_wait(a_full, 0, abort_flag);
            if (!ok) fail();
            const uint32_t a_base = smem_u32(sA);
            for (int i = 0; ok && i < nt; ++i) {
                const int buf = i & 1;
                if (!mbar_wait(&t_empty[buf], ((i >> 1) & 1) ^ 1, abort_flag)) { fail(); break; }
                for (int kb = 0; kb < KB; ++kb) {
                    const int g = i * KB + kb, s = g % NST;
                    if (!mbar_wait(&full[s], (g / NST) & 1, abort_flag)) { fail(); ok = false; break; }
                    tc_fence_after();
                    const uint32_t b_base = smem_u32(sB + static_cast<size_t>(s) * kTileBytes);
                    const int k4 = min(4, a.ksteps - kb * 4);   // 32-byte K steps in this block
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt) {
                        const uint32_t d_tmem = tmem + (buf * MT + mt) * kBlockN;
                        const uint32_t am = a_base + (mt * KB + kb) * kTileBytes;
                        for (int ks = 0; ks < k4; ++ks)
                            mma<PREC>(d_tmem, sdesc(am + ks * 32), sdesc(b_base + ks * 32), id,
                                      (kb | ks) ? 1u : 0u);
                    }
                    tc_commit(&empty[s]);
                }
                if (!ok) break;
                tc_commit(&t_full[buf]);
            }
            tc_commit(drain);   // arrives once every MMA issued above has completed
            mbar_wait(drain, 0, nullptr);
        }
        __syncwarp();
    } else {
        // -------------------------------------------------------- epilogue
        const int et = threadIdx.x - 64;            // 0 .. kEpi-1
        const int mt = et / 128;
        const int quarter = warp & 3;               // the TMEM lanes this warp may access
        const int row = quarter * 32 + lane;
        const int64_t q = q0 + mt * kBlockM + row;
        const bool active = q < a.n;
        const uint32_t lane_addr = tmem + (static_cast<uint32_t>(quarter * 32) << 16);
        float* st = stage + et * 32;
        const int sw = et & 7;                      // bank swizzle of this thread's slot
        uint64_t* list = nullptr;
        uint32_t* gout = nullptr;
        if (PILOT) gout = a.gmax + q * a.G + static_cast<int64_t>(split) * a.spt * 4;
        else list = a.lists + (q * a.S + split) * static_cast<int64_t>(a.cap);
        int cnt = 0;
        for (int i = 0; i < nt; ++i) {
            const int buf = i & 1;
            const bool ok = mbar_wait(&t_full[buf], (i >> 1) & 1, abort_flag);
            if (!__all_sync(0xffffffffu, ok)) { fail(); break; }
            tc_fence_after();
            const int64_t jt = r_begin + static_cast<int64_t>(i) * stride * kBlockN;
#pragma unroll 1
            for (int ch = 0; ch < kBlockN / 32; ++ch) {
                uint32_t r[32];
                __syncwarp();
                tmem_ld32u(lane_addr + (buf * MT + mt) * kBlockN + ch * 32, r);
                if (ch == kBlockN / 32 - 1) {
                    tc_fence_before();
                    mbar_arrive(&t_empty[buf]);
                }
                const int64_t j0 = jt + ch * 32;
                const int64_t left = r_end - j0;
                const int nvalid = left <= 0 ? 0 : (left >= 32 ? 32 : static_cast<int>(left));
                if (PILOT) {
                    float mx = __int_as_float(0xff800000);   // -inf
#pragma unroll
                    for (int u = 0; u < 32; ++u)
                        mx = fmaxf(mx, u < nvalid ? __uint_as_float(r[u]) : __int_as_float(0xff800000));
                    if (active && nvalid > 0) gout[i * 4 + ch] = ord_f32(mx);
                } else {
                    uint32_t sm = 0;
#pragma unroll
                    for (int u = 0; u < 32; ++u) sm = __funnelshift_l(r[u], sm, 1);
                    // bit 31-u is the sign of element u; a pass is acc >= 0
                    uint32_t hits = a.append_all ? 0xffffffffu : ~sm;
                    hits &= nvalid == 0 ? 0u : (0xffffffffu << (32 - nvalid));
                    if (!active) hits = 0;
                    if (hits) {
#pragma unroll
                        for (int g = 0; g < 8; ++g)
                            reinterpret_cast<uint4*>(st)[g ^ sw] =
                                make_uint4(r[4 * g], r[4 * g + 1], r[4 * g + 2], r[4 * g + 3]);
                        while (hits) {
                            const int u = __clz(hits);
                            hits &= ~(0x80000000u >> u);
                            const float v = st[(((u >> 2) ^ sw) << 2) | (u & 3)];
                            if (cnt < a.cap) list[cnt] = make_key(-v, static_cast<uint32_t>(j0 + u));
                            ++cnt;
                        }
                    }
                }
            }
        }
        if (!PILOT && active) a.counts[q * a.S + split] = cnt;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// ------------------------------------------------ operand preparation kernels
template <int PREC>
__device__ __forceinline__ void put(void* row, int t, float v) {
    if (PREC == kBF16) {
        reinterpret_cast<__nv_bfloat16*>(row)[t] = __float2bfloat16_rn(v);
    } else {
        uint32_t b;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(b) : "f"(v));
        reinterpret_cast<uint32_t*>(row)[t] = b;
    }
}
template <int PREC>
__device__ __forceinline__ float lowp_round(float v) {
    if (PREC == kBF16) return __bfloat162float(__float2bfloat16_rn(v));
    uint32_t b;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(b) : "f"(v));
    return __uint_as_float(b);
}

// One warp per row.  REF: [x, -nr_hi/2, -nr_lo/2, 1, 1, 0..] and the float32
// squared norm; QUERY: [x, 1, 1, 0, 0, 0..] (threshold words filled later).
template <int PREC, bool REF>
__global__ void prepare_kernel(const float* __restrict__ X, int64_t rows, int32_t d, int32_t kp,
                               void* __restrict__ out, float* __restrict__ norms) {
    const int64_t r = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (r >= rows) return;
    const float* x = X + r * d;
    const size_t elt = (PREC == kBF16) ? 2 : 4;
    void* row = static_cast<unsigned char*>(out) + static_cast<size_t>(r) * kp * elt;
    float nr = 0.f;
    if (REF) {
        for (int t = lane; t < d; t += 32) nr = fmaf(x[t], x[t], nr);
        for (int o = 16; o > 0; o >>= 1) nr += __shfl_xor_sync(0xffffffffu, nr, o);
        if (lane == 0 && norms) norms[r] = nr;
    }
    const float h = -0.5f * nr;
    const float hi = lowp_round<PREC>(h);
    const float lo = lowp_round<PREC>(h - hi);
    for (int t = lane; t < kp; t += 32) {
        float v = 0.f;
        if (t < d) v = x[t];
        else if (t == d) v = REF ? hi : 1.f;
        else if (t == d + 1) v = REF ? lo : 1.f;
        else if (t == d + 2 || t == d + 3) v = REF ? 1.f : 0.f;
        put<PREC>(row, t, v);
    }
}

// One warp per query: the cprime-th largest group maximum of the pilot becomes
// the query's threshold, written into its threshold words with a margin that
// covers the rounding difference between the pilot and filter products.
template <int PREC>
__global__ void threshold_kernel(const uint32_t* __restrict__ gmax, int64_t n, int32_t G,
                                 int32_t cprime, int32_t d, int32_t kp, void* __restrict__ Q_lp) {
    extern __shared__ uint32_t vals[];
    const int wib = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t q = static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + wib;
    if (q >= n) return;
    uint32_t* v = vals + wib * G;
    for (int g = lane; g < G; g += 32) v[g] = gmax[q * G + g];
    __syncwarp();
    uint32_t best = 0, least = 0xffffffffu;
    for (int g = lane; g < G; g += 32)
        if (v[g] != 0) least = min(least, v[g]);
    for (int o = 16; o > 0; o >>= 1) least = min(least, __shfl_xor_sync(0xffffffffu, least, o));
    for (int rep = 0; rep < cprime; ++rep) {
        uint32_t mx = 0;
        int at = -1;
        for (int g = lane; g < G; g += 32)
            if (v[g] > mx) { mx = v[g]; at = g; }
        uint32_t wmx = mx;
        for (int o = 16; o > 0; o >>= 1) wmx = max(wmx, __shfl_xor_sync(0xffffffffu, wmx, o));
        if (wmx == 0) break;
        const unsigned own = __ballot_sync(0xffffffffu, mx == wmx && at >= 0);
        if (lane == __ffs(own) - 1) v[at] = 0;
        __syncwarp();
        best = wmx;
    }
    if (best == 0) best = least;   // fewer groups than cprime: weakest group seen
    const float t_acc = unord_f32(best);
    const float tcol = -t_acc + 1e-3f * (1.f + fabsf(t_acc));
    const float hi = lowp_round<PREC>(tcol);
    const float lo = lowp_round<PREC>(tcol - hi);
    if (lane == 0) {
        const size_t elt = (PREC == kBF16) ? 2 : 4;
        void* row = static_cast<unsigned char*>(Q_lp) + static_cast<size_t>(q) * kp * elt;
        put<PREC>(row, d + 2, hi);
        put<PREC>(row, d + 3, lo);
    }
}

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

// rows x kp operand; box = 128 bytes of K x 128 rows; 128-byte swizzle; zero fill.
bool make_map(CUtensorMap* map, const void* base, int64_t rows, int kp, int prec) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const int elt = (prec == kBF16) ? 2 : 4;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(kp), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(kp) * elt};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kAtomBytes / elt), static_cast<cuuint32_t>(kBlockM)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map,
                    prec == kBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                    2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int PREC, int MT, bool PILOT>
cudaError_t launch_kernel(const TcPlan& p, const CUtensorMap& mq, const CUtensorMap& mr,
                          const TcArgs& a, cudaStream_t st) {
    auto kern = tc_kernel<PREC, MT, PILOT>;
    const size_t smem = tc_smem_bytes(MT, p.kb, p.stages, PILOT);
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    dim3 grid(static_cast<unsigned>((a.n + kBlockM * MT - 1) / (kBlockM * MT)),
              static_cast<unsigned>(a.S));
    kern<<<grid, 64 + 128 * MT, smem, st>>>(mq, mr, a);
    return cudaGetLastError();
}

template <bool PILOT>
cudaError_t dispatch(const TcPlan& p, int prec, const CUtensorMap& mq, const CUtensorMap& mr,
                     const TcArgs& a, cudaStream_t st) {
    if (prec == kBF16)
        return p.mt == 2 ? launch_kernel<kBF16, 2, PILOT>(p, mq, mr, a, st)
                         : launch_kernel<kBF16, 1, PILOT>(p, mq, mr, a, st);
    return p.mt == 2 ? launch_kernel<kTF32, 2, PILOT>(p, mq, mr, a, st)
                     : launch_kernel<kTF32, 1, PILOT>(p, mq, mr, a, st);
}

TcArgs base_args(const TcPlan& p, int64_t n, int64_t m, int32_t* error_flag) {
    TcArgs a{};
    a.n = n;
    a.m = m;
    a.kb = p.kb;
    a.ksteps = p.ksteps;
    a.stages = p.stages;
    a.chunk = p.chunk;
    a.S = p.S;
    a.stride = p.stride;
    a.spt = p.spt;
    a.G = p.G;
    a.cap = p.cap;
    a.append_all = p.pilot ? 0 : 1;
    a.error_flag = error_flag;
    return a;
}

}  // namespace

int tc_padded_dim(int32_t d, int prec) {
    const int step = (prec == kBF16) ? 16 : 8;   // 32 bytes: one MMA K step
    return (d + kAugCols + step - 1) / step * step;
}

TcPlan tc_plan(int64_t n, int64_t m, int32_t kp, int prec, int32_t c, int num_sms) {
    TcPlan p{};
    const int elt = (prec == kBF16) ? 2 : 4;
    p.kb = (kp * elt + kAtomBytes - 1) / kAtomBytes;
    p.ksteps = kp * elt / 32;
    p.stages = 0;
    // two query tiles per CTA when the ring still holds two reference tiles
    for (int mt = 2; mt >= 1 && p.stages == 0; --mt) {
        const int need = (mt == 2) ? 2 * p.kb : 2;
        for (int s = kMaxStages; s >= need; --s) {
            if (tc_smem_bytes(mt, p.kb, s, false) <= kSmemLimit) {
                p.mt = mt;
                p.stages = s;
                break;
            }
        }
    }
    if (p.stages == 0) return p;   // operand rows too long for shared memory
    const int64_t qtiles = (n + kBlockM * p.mt - 1) / (kBlockM * p.mt);
    // reference splits: the fewest whose CTAs fill at least 85% of the last wave
    int64_t max_s = m / (16 * kBlockN);
    if (max_s < 1) max_s = 1;
    if (max_s > 64) max_s = 64;
    int S = 1;
    double best = 0.0;
    for (int s = 1; s <= max_s; ++s) {
        const int64_t ctas = qtiles * s;
        const int64_t waves = (ctas + num_sms - 1) / num_sms;
        const double eff = static_cast<double>(ctas) / (static_cast<double>(waves) * num_sms);
        if (eff > best + 1e-9) { best = eff; S = s; }
        if (eff >= 0.85) break;
    }
    int64_t chunk = (m + S - 1) / S;
    chunk = (chunk + kBlockN - 1) / kBlockN * kBlockN;
    S = static_cast<int>((m + chunk - 1) / chunk);
    p.S = S;
    p.chunk = chunk;
    // pilot sampling: every stride-th tile, at most ~1024 groups per query
    const int64_t tiles_total = (m + kBlockN - 1) / kBlockN;
    int stride = 16;
    while (tiles_total * 4 / stride > 1024) stride *= 2;
    const int tps = static_cast<int>(chunk / kBlockN);
    p.stride = stride;
    p.spt = (tps + stride - 1) / stride;
    p.G = S * p.spt * 4;
    const double lambda = static_cast<double>(c) / stride;
    p.cprime = static_cast<int>(std::ceil(lambda + 6.0 * std::sqrt(lambda) + 4.0));
    p.pilot = (p.G >= 2 * p.cprime) ? 1 : 0;
    if (p.pilot) {
        const int64_t expect = static_cast<int64_t>(p.cprime) * stride;
        int64_t cap = (2 * expect + 255) / S + 128;
        p.cap = static_cast<int32_t>((cap + 31) / 32 * 32);
    } else {
        p.cap = static_cast<int32_t>(chunk);
    }
    p.smem_filter = tc_smem_bytes(p.mt, p.kb, p.stages, false);
    return p;
}

cudaError_t launch_prepare_ref(const float* R, int64_t m, int32_t d, int32_t kp, int prec,
                               void* R_lp, float* norms, cudaStream_t st, int* launches) {
    const unsigned grid = static_cast<unsigned>((m * 32 + 255) / 256);
    if (prec == kBF16) prepare_kernel<kBF16, true><<<grid, 256, 0, st>>>(R, m, d, kp, R_lp, norms);
    else prepare_kernel<kTF32, true><<<grid, 256, 0, st>>>(R, m, d, kp, R_lp, norms);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_prepare_query(const float* Q, int64_t n, int32_t d, int32_t kp, int prec,
                                 void* Q_lp, cudaStream_t st, int* launches) {
    const unsigned grid = static_cast<unsigned>((n * 32 + 255) / 256);
    if (prec == kBF16) prepare_kernel<kBF16, false><<<grid, 256, 0, st>>>(Q, n, d, kp, Q_lp, nullptr);
    else prepare_kernel<kTF32, false><<<grid, 256, 0, st>>>(Q, n, d, kp, Q_lp, nullptr);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_tc_pilot(const TcPlan& p, const void* Q_lp, int64_t n, const void* R_lp, int64_t m,
                            int32_t kp, int prec, uint32_t* gmax, int32_t* error_flag, cudaStream_t st,
                            int* launches) {
    CUtensorMap mq, mr;
    if (!make_map(&mq, Q_lp, n, kp, prec) || !make_map(&mr, R_lp, m, kp, prec))
        return cudaErrorInvalidValue;
    cudaError_t err = cudaMemsetAsync(gmax, 0, static_cast<size_t>(n) * p.G * 4, st);
    if (err != cudaSuccess) return err;
    TcArgs a = base_args(p, n, m, error_flag);
    a.gmax = gmax;
    if (launches) ++*launches;
    return dispatch<true>(p, prec, mq, mr, a, st);
}

cudaError_t launch_tc_threshold(const TcPlan& p, const uint32_t* gmax, int64_t n, int32_t d,
                                int32_t kp, int prec, void* Q_lp, cudaStream_t st, int* launches) {
    const int wpb = 4;
    const size_t smem = static_cast<size_t>(wpb) * p.G * 4;
    const unsigned grid = static_cast<unsigned>((n + wpb - 1) / wpb);
    if (prec == kBF16)
        threshold_kernel<kBF16><<<grid, wpb * 32, smem, st>>>(gmax, n, p.G, p.cprime, d, kp, Q_lp);
    else
        threshold_kernel<kTF32><<<grid, wpb * 32, smem, st>>>(gmax, n, p.G, p.cprime, d, kp, Q_lp);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_tc_filter(const TcPlan& p, const void* Q_lp, int64_t n, const void* R_lp, int64_t m,
                             int32_t kp, int prec, uint64_t* lists, int32_t* counts,
                             int32_t* error_flag, cudaStream_t st, int* launches) {
    CUtensorMap mq, mr;
    if (!make_map(&mq, Q_lp, n, kp, prec) || !make_map(&mr, R_lp, m, kp, prec))
        return cudaErrorInvalidValue;
    TcArgs a = base_args(p, n, m, error_flag);
    a.stride = 1;
    a.lists = lists;
    a.counts = counts;
    if (launches) ++*launches;
    return dispatch<false>(p, prec, mq, mr, a, st);
}

}  // namespace knn
