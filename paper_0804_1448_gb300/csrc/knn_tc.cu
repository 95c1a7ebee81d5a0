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
//                 a ring of single-K-block shared-memory stages (128-byte swizzle);
//   warp 1        MMA issuer: per reference tile and query tile, kp*elt/32
//                 tcgen05.mma into one of two TMEM accumulators per query tile;
//                 tcgen05.commit frees the smem stage and publishes the tile;
//   warps 2..     epilogue, 8 per query tile: warp w may read the TMEM lanes
//                 32*(w%4)..+31, so thread t of warp w owns query row
//                 32*(w%4)+t; the two warps sharing a lane quarter split the
//                 four 32-column slices of each tile between them.
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
// Floats per thread in the hit-staging area: a whole 32-value slice + pad, or
// (when shared memory is short) 16 values + pad; either stride keeps eight
// lanes' 16-byte stores on distinct banks.
constexpr int kStageFull = 36;
constexpr int kStageHalf = 20;

struct TcArgs {
    int64_t n, m;
    int32_t kb;           // 128-byte K blocks per operand row (row pitch = kb * 128 bytes)
    int32_t ksteps;       // 32-byte MMA K steps that carry data
    int32_t rb;           // references per pipeline stage (128 or 256): rb/128 MMA tiles
    int32_t kbs;          // K blocks per stage: kb (whole rows) or 1 (then rb = 128)
    int32_t stages;
    int64_t chunk;        // references per split (multiple of rb)
    int32_t S;
    int32_t stride;       // pilot: every stride-th stage of a split
    int32_t spt;          // pilot: sampled-stage slots per split
    int32_t G;            // pilot: group maxima per query (S * spt * rb / 32)
    uint32_t* gmax;       // pilot: [n][G] order-mapped maxima, 0 = no group
    uint64_t* lists;      // filter: [n][S][2][cap], one list per epilogue half
    int32_t* counts;      // filter: [n][S][2] (may exceed cap: overflow)
    int32_t cap;
    int32_t append_all;   // filter: every valid reference passes
    int32_t stage_half;   // filter: stage hit values per 16-element half slice
    int32_t* error_flag;
};

// A: mt query tiles of kb K blocks (resident); B: a ring of `stages` boxes of
// rb references x kbs K blocks; staging of hit values (filter only).
__host__ __device__ constexpr size_t tc_smem_bytes(int mt, int kb, int rb, int kbs, int stages,
                                                   bool pilot, bool half_stage = false) {
    return 1024 + static_cast<size_t>(kTileBytes) * mt * kb +
           static_cast<size_t>(rb) * kAtomBytes * kbs * stages +
           (pilot ? 0 : static_cast<size_t>(256) * mt * (half_stage ? kStageHalf : kStageFull) * 4) +
           512;
}

// Append one passing reference to a hit list.  key = (order of -acc, index):
// a threshold pass has acc >= +0, so the order of -acc is ~bits(acc) without
// its sign bit; without a threshold acc may have either sign.
__device__ __forceinline__ void append(uint64_t* list, int& cnt, int cap, uint32_t vb, uint32_t j,
                                       int append_all) {
    const uint32_t o = append_all ? ord_f32(-__uint_as_float(vb)) : (~vb & 0x7fffffffu);
    if (cnt < cap) list[cnt] = (static_cast<uint64_t>(o) << 32) | j;
    ++cnt;
}

// MMAs of one 128-byte K block of one reference tile for all MT query tiles.
// Fully unrolled over the four 32-byte K steps (a runtime guard skips steps
// past the data): issue from the single MMA thread must keep pace with the
// tensor core, and a loop with runtime bounds halves the issue rate.
template <int PREC, int MT>
__device__ __forceinline__ void issue_kblock(uint32_t d_tmem, uint32_t a_kb, uint32_t a_mt_stride,
                                             uint32_t b_kb, int k4, bool first, uint32_t id) {
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            if (ks < k4)
                mma<PREC>(d_tmem + mt * kBlockN, sdesc(a_kb + mt * a_mt_stride + ks * 32),
                          sdesc(b_kb + ks * 32), id, (first && ks == 0) ? 0u : 1u);
        }
    }
}

// KBT > 0: whole-K stages of exactly KBT K blocks (compile-time, unrolled);
// KBT == 0: any K-block count and either stage layout (loops over K blocks).
template <int PREC, int MT, bool PILOT, int KBT>
__global__ void __launch_bounds__(64 + 256 * MT, 1)
tc_kernel(const __grid_constant__ CUtensorMap tmap_q, const __grid_constant__ CUtensorMap tmap_r,
          TcArgs a) {
    constexpr int kEpi = 256 * MT;             // epilogue threads: two per query row
    constexpr uint32_t kTmemCols = 256 * MT;   // two 128-column accumulators per query tile
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);

    const int KB = KBT > 0 ? KBT : a.kb, KBS = KBT > 0 ? KBT : a.kbs;
    const int NST = a.stages, RB = a.rb, TPS = a.rb / kBlockN;
    const int SPT = KB / KBS;                   // stages per reference tile (1, or KB when KBS = 1)
    const size_t stage_bytes = static_cast<size_t>(RB) * kAtomBytes * KBS;
    unsigned char* sA = smem;
    unsigned char* sB = sA + static_cast<size_t>(MT) * KB * kTileBytes;
    float* stage = reinterpret_cast<float*>(sB + NST * stage_bytes);
    const int stride_st = a.stage_half ? kStageHalf : kStageFull;
    uint64_t* bars = reinterpret_cast<uint64_t*>(stage + (PILOT ? 0 : kEpi * stride_st));
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
    const int stages_all = static_cast<int>((r_end - r_begin + RB - 1) / RB);
    const int stride = PILOT ? a.stride : 1;
    const int ng = (stages_all + stride - 1) / stride;   // stages this CTA processes
    const int nt = ng * TPS;                             // MMA tiles

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
        // one 3-D box per operand load: (128 bytes of K) x rows x all K blocks
        if (lane == 0) {
            mbar_expect_tx(a_full, MT * KB * kTileBytes);
            for (int mt = 0; mt < MT; ++mt)
                tma_load_3d(sA + static_cast<size_t>(mt) * KB * kTileBytes, &tmap_q, a_full, 0,
                            static_cast<int>(q0 + mt * kBlockM), 0);
            int issued = 0;   // stage h = g * SPT + kb: reference rows of g, K blocks kb..
            for (int h = 0; h < ng * SPT; ++h) {
                const int g = h / SPT, z = (h % SPT) * KBS, s = h % NST;
                if (!mbar_wait(&empty[s], ((h / NST) & 1) ^ 1, abort_flag)) { fail(); break; }
                mbar_expect_tx(&full[s], static_cast<uint32_t>(stage_bytes));
                const int y = static_cast<int>(r_begin + static_cast<int64_t>(g) * stride * RB);
                tma_load_3d(sB + s * stage_bytes, &tmap_r, &full[s], 0, y, z);
                issued = h + 1;
            }
            mbar_wait(a_full, 0, nullptr);   // drain: every issued copy has landed
            for (int h = (issued > NST ? issued - NST : 0); h < issued; ++h)
                mbar_wait(&full[h % NST], (h / NST) & 1, nullptr);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t id = idesc(PREC == kBF16 ? 1 : 2, kBlockM, kBlockN);
            bool ok = mbar_wait(a_full, 0, abort_flag);
            if (!ok) fail();
            const uint32_t a_base = smem_u32(sA);
            if (SPT == 1) {
                // whole-K stages: stage g holds TPS tiles of 128 references
                for (int g = 0; ok && g < ng; ++g) {
                    const int s = g % NST;
                    if (!mbar_wait(&full[s], (g / NST) & 1, abort_flag)) { fail(); break; }
                    const uint32_t b_stage = smem_u32(sB + s * stage_bytes);
                    for (int t2 = 0; t2 < TPS; ++t2) {
                        const int i = g * TPS + t2, buf = i & 1;
                        if (!mbar_wait(&t_empty[buf], ((i >> 1) & 1) ^ 1, abort_flag)) {
                            fail();
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d_tmem = tmem + buf * MT * kBlockN;
                        const uint32_t b_tile = b_stage + t2 * kTileBytes;
                        if (KBT > 0) {
#pragma unroll
                            for (int kb = 0; kb < (KBT > 0 ? KBT : 1); ++kb)
                                issue_kblock<PREC, MT>(d_tmem, a_base + kb * kTileBytes, KB * kTileBytes,
                                                       b_tile + kb * RB * kAtomBytes,
                                                       a.ksteps - kb * 4, kb == 0, id);
                        } else {
                            for (int kb = 0; kb < KB; ++kb)
                                issue_kblock<PREC, MT>(d_tmem, a_base + kb * kTileBytes, KB * kTileBytes,
                                                       b_tile + kb * RB * kAtomBytes,
                                                       a.ksteps - kb * 4, kb == 0, id);
                        }
                        tc_commit(&t_full[buf]);
                    }
                    tc_commit(&empty[s]);   // the stage is free once these MMAs complete
                }
            } else {
                // one K block per stage: tile g takes stages g*KB .. g*KB+KB-1
                for (int g = 0; ok && g < ng; ++g) {
                    const int buf = g & 1;
                    if (!mbar_wait(&t_empty[buf], ((g >> 1) & 1) ^ 1, abort_flag)) { fail(); break; }
                    for (int kb = 0; kb < KB; ++kb) {
                        const int h = g * KB + kb, s = h % NST;
                        if (!mbar_wait(&full[s], (h / NST) & 1, abort_flag)) {
                            fail();
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        issue_kblock<PREC, MT>(tmem + buf * MT * kBlockN, a_base + kb * kTileBytes,
                                               KB * kTileBytes, smem_u32(sB + s * stage_bytes),
                                               a.ksteps - kb * 4, kb == 0, id);
                        tc_commit(&empty[s]);
                    }
                    if (!ok) break;
                    tc_commit(&t_full[buf]);
                }
            }
            tc_commit(drain);   // arrives once every MMA issued above has completed
            mbar_wait(drain, 0, nullptr);
        }
        __syncwarp();
    } else {
        // -------------------------------------------------------- epilogue
        const int et = threadIdx.x - 64;            // 0 .. kEpi-1
        const int ew = et / 32;
        const int mt = (ew / 4) % MT;
        const int half = ew / (4 * MT);             // slices 2*half, 2*half+1 of every tile
        const int quarter = warp & 3;               // the TMEM lanes this warp may access
        const int row = quarter * 32 + lane;
        const int64_t q = q0 + mt * kBlockM + row;
        const bool active = q < a.n;
        const uint32_t lane_addr = tmem + (static_cast<uint32_t>(quarter * 32) << 16);
        float* st = stage + et * stride_st;
        const int gpt = RB / 32;                    // groups of 32 references per stage
        uint64_t* list = nullptr;
        uint32_t* gout = nullptr;
        if (PILOT) gout = a.gmax + q * a.G + static_cast<int64_t>(split) * a.spt * gpt;
        // each half-warp owns its own list: (query, split, half)
        else list = a.lists + ((q * a.S + split) * 2 + half) * static_cast<int64_t>(a.cap);
        int cnt = 0;
        for (int i = 0; i < nt; ++i) {
            const int buf = i & 1, g = i / TPS, t2 = i % TPS;
            const bool ok = mbar_wait(&t_full[buf], (i >> 1) & 1, abort_flag);
            if (!__all_sync(0xffffffffu, ok)) { fail(); break; }
            tc_fence_after();
            const int64_t jt = r_begin + static_cast<int64_t>(g) * stride * RB + t2 * kBlockN;
            // this warp's two 32-column slices; the second loads while the
            // first is processed
            uint32_t ra[32], rb[32];
            const uint32_t col0 = lane_addr + (buf * MT + mt) * kBlockN + half * 64;
            __syncwarp();
            tmem_ld32u_async(col0, ra);
#pragma unroll
            for (int sl = 0; sl < 2; ++sl) {
                const int ch = 2 * half + sl;
                uint32_t (&r)[32] = sl ? rb : ra;
                tmem_wait_ld(r);
                if (sl == 0) {
                    tmem_ld32u_async(col0 + 32, rb);
                } else {
                    tc_fence_before();
                    mbar_arrive(&t_empty[buf]);   // both slices of this buffer are in registers
                }
                const int64_t j0 = jt + ch * 32;
                const int64_t left = r_end - j0;
                const int nvalid = left <= 0 ? 0 : (left >= 32 ? 32 : static_cast<int>(left));
                if (PILOT) {
                    float v[32];
#pragma unroll
                    for (int u = 0; u < 32; ++u)
                        v[u] = u < nvalid ? __uint_as_float(r[u]) : __int_as_float(0xff800000);
#pragma unroll
                    for (int w2 = 16; w2 > 0; w2 >>= 1)
#pragma unroll
                        for (int u = 0; u < w2; ++u) v[u] = fmaxf(v[u], v[u + w2]);
                    if (active && nvalid > 0) gout[g * gpt + t2 * 4 + ch] = ord_f32(v[0]);
                } else {
                    // sign bits, bit 31-u for element u, as four independent chains
                    uint32_t m4[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                    for (int u = 0; u < 8; ++u)
#pragma unroll
                        for (int h = 0; h < 4; ++h) m4[h] = __funnelshift_l(r[8 * h + u], m4[h], 1);
                    const uint32_t sm = (m4[0] << 24) | (m4[1] << 16) | (m4[2] << 8) | m4[3];
                    // a pass is acc >= 0; bit u of `hits` is element u after the reversal
                    uint32_t hits = __brev(a.append_all ? 0xffffffffu : ~sm);
                    hits &= nvalid >= 32 ? 0xffffffffu : ((1u << nvalid) - 1u);
                    if (!active) hits = 0;
                    // the append loop reads the hit values with a dynamic index, which
                    // registers do not allow: they go through shared memory first
                    if (!a.stage_half) {
                        if (hits) {
#pragma unroll
                            for (int h = 0; h < 8; ++h)
                                reinterpret_cast<uint4*>(st)[h] =
                                    make_uint4(r[4 * h], r[4 * h + 1], r[4 * h + 2], r[4 * h + 3]);
                            const uint32_t jb = static_cast<uint32_t>(j0);
                            do {
                                const int u = __ffs(hits) - 1;
                                hits &= hits - 1;
                                append(list, cnt, a.cap, __float_as_uint(st[u]), jb + u, a.append_all);
                            } while (hits);
                        }
                    } else {
#pragma unroll
                        for (int hf = 0; hf < 2; ++hf) {
                            uint32_t hh = (hits >> (16 * hf)) & 0xffffu;
                            if (hh) {
#pragma unroll
                                for (int h = 0; h < 4; ++h)
                                    reinterpret_cast<uint4*>(st)[h] =
                                        make_uint4(r[16 * hf + 4 * h], r[16 * hf + 4 * h + 1],
                                                   r[16 * hf + 4 * h + 2], r[16 * hf + 4 * h + 3]);
                                const uint32_t jb = static_cast<uint32_t>(j0) + 16 * hf;
                                do {
                                    const int u = __ffs(hh) - 1;
                                    hh &= hh - 1;
                                    append(list, cnt, a.cap, __float_as_uint(st[u]), jb + u,
                                           a.append_all);
                                } while (hh);
                            }
                        }
                    }
                    __syncwarp();
                }
            }
        }
        if (!PILOT && active) a.counts[(q * a.S + split) * 2 + half] = cnt;
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

// rows x kp operand seen as 3-D: (128 bytes of K) x rows x K blocks, so one box
// brings box_rows rows with all their K blocks, laid out block-major
// ([K block][row][128 bytes], 128-byte swizzle) as the MMA descriptors expect.
// Rows outside the tensor read as zero.
bool make_map(CUtensorMap* map, const void* base, int64_t rows, int kp, int prec, int box_rows,
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

template <int PREC, int MT, bool PILOT, int KBT>
cudaError_t launch_kernel(const TcPlan& p, const CUtensorMap& mq, const CUtensorMap& mr,
                          const TcArgs& a, cudaStream_t st) {
    auto kern = tc_kernel<PREC, MT, PILOT, KBT>;
    const size_t smem = tc_smem_bytes(MT, p.kb, p.rb, p.kbs, p.stages, PILOT, p.stage_half != 0);
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    dim3 grid(static_cast<unsigned>((a.n + kBlockM * MT - 1) / (kBlockM * MT)),
              static_cast<unsigned>(a.S));
    kern<<<grid, 64 + 256 * MT, smem, st>>>(mq, mr, a);
    return cudaGetLastError();
}

template <int PREC, int MT, bool PILOT>
cudaError_t dispatch_kb(const TcPlan& p, const CUtensorMap& mq, const CUtensorMap& mr,
                        const TcArgs& a, cudaStream_t st) {
    if (p.kbs == p.kb) {   // whole-K stages: unrolled issue for the common row lengths
        switch (p.kb) {
            case 1: return launch_kernel<PREC, MT, PILOT, 1>(p, mq, mr, a, st);
            case 2: return launch_kernel<PREC, MT, PILOT, 2>(p, mq, mr, a, st);
            case 3: return launch_kernel<PREC, MT, PILOT, 3>(p, mq, mr, a, st);
            case 4: return launch_kernel<PREC, MT, PILOT, 4>(p, mq, mr, a, st);
            default: break;
        }
    }
    return launch_kernel<PREC, MT, PILOT, 0>(p, mq, mr, a, st);
}

template <bool PILOT>
cudaError_t dispatch(const TcPlan& p, int prec, const CUtensorMap& mq, const CUtensorMap& mr,
                     const TcArgs& a, cudaStream_t st) {
    if (prec == kBF16)
        return p.mt == 2 ? dispatch_kb<kBF16, 2, PILOT>(p, mq, mr, a, st)
                         : dispatch_kb<kBF16, 1, PILOT>(p, mq, mr, a, st);
    return p.mt == 2 ? dispatch_kb<kTF32, 2, PILOT>(p, mq, mr, a, st)
                     : dispatch_kb<kTF32, 1, PILOT>(p, mq, mr, a, st);
}

TcArgs base_args(const TcPlan& p, int64_t n, int64_t m, int32_t* error_flag) {
    TcArgs a{};
    a.n = n;
    a.m = m;
    a.kb = p.kb;
    a.ksteps = p.ksteps;
    a.rb = p.rb;
    a.kbs = p.kbs;
    a.stages = p.stages;
    a.chunk = p.chunk;
    a.S = p.S;
    a.stride = p.stride;
    a.spt = p.spt;
    a.G = p.G;
    a.cap = p.cap;
    a.append_all = p.pilot ? 0 : 1;
    a.stage_half = p.stage_half;
    a.error_flag = error_flag;
    return a;
}

}  // namespace

int tc_padded_dim(int32_t d, int prec) {
    const int step = (prec == kBF16) ? 64 : 32;   // whole 128-byte K blocks per row
    return (d + kAugCols + step - 1) / step * step;
}

TcPlan tc_plan(int64_t n, int64_t m, int32_t d, int32_t kp, int prec, int32_t c, int num_sms) {
    TcPlan p{};
    const int elt = (prec == kBF16) ? 2 : 4;
    const int kstep = 32 / elt;                    // elements per MMA K step
    p.kb = kp * elt / kAtomBytes;
    p.ksteps = (d + kAugCols + kstep - 1) / kstep;
    p.stages = 0;
    // prefer two query tiles per CTA and whole-K 256-reference stages, then
    // shrink; single-K-block stages (more TMA boxes) only when rows are long
    // {query tiles, references per stage, one K block per stage, half-slice staging}
    const int shapes[10][4] = {{2, 256, 0, 0}, {2, 128, 0, 0}, {1, 256, 0, 0}, {1, 128, 0, 0},
                               {2, 128, 0, 1}, {1, 128, 0, 1}, {2, 128, 1, 0}, {1, 128, 1, 0},
                               {2, 128, 1, 1}, {1, 128, 1, 1}};
    // whole-K 256-reference stages need a third stage to hide the TMA latency;
    // with 128-reference stages two boxes per tile pair are already in flight
    for (int si = 0; si < 10 && p.stages == 0; ++si) {
        const int kbs = shapes[si][2] ? 1 : p.kb;
        const int smax = shapes[si][2] ? 12 : kMaxStages;
        const int smin = (!shapes[si][2] && shapes[si][1] == 256) ? 3 : 2;
        for (int s = smax; s >= smin; --s) {
            if (tc_smem_bytes(shapes[si][0], p.kb, shapes[si][1], kbs, s, false, shapes[si][3] != 0) <=
                kSmemLimit) {
                p.mt = shapes[si][0];
                p.rb = shapes[si][1];
                p.kbs = kbs;
                p.stage_half = shapes[si][3];
                p.stages = s;
                break;
            }
        }
    }
    if (p.stages == 0) return p;   // operand rows too long for shared memory
    const int64_t qtiles = (n + kBlockM * p.mt - 1) / (kBlockM * p.mt);
    // reference splits: the fewest whose CTAs fill at least 85% of the last wave
    int64_t max_s = m / (8 * p.rb);
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
    chunk = (chunk + p.rb - 1) / p.rb * p.rb;
    S = static_cast<int>((m + chunk - 1) / chunk);
    p.S = S;
    p.chunk = chunk;
    // pilot sampling: every stride-th stage, at most ~1024 groups per query
    const int gps = p.rb / 32;                     // groups of 32 references per stage
    const int64_t stages_total = (m + p.rb - 1) / p.rb;
    int stride = 2048 / p.rb;                      // one stage in 16 tiles of 128
    while (stages_total * gps / stride > 1024) stride *= 2;
    const int sps = static_cast<int>(chunk / p.rb);
    p.stride = stride;
    p.spt = (sps + stride - 1) / stride;
    p.G = S * p.spt * gps;
    const double frac = static_cast<double>(p.rb) / (static_cast<double>(stride) * p.rb);
    const double lambda = static_cast<double>(c) * frac;
    p.cprime = static_cast<int>(std::ceil(lambda + 6.0 * std::sqrt(lambda) + 4.0));
    p.pilot = (p.G >= 2 * p.cprime) ? 1 : 0;
    // list capacity per (query, split, half): twice the expected hits plus slack
    if (p.pilot) {
        const int64_t expect = static_cast<int64_t>(p.cprime) * stride;
        int64_t cap = (2 * expect + 255) / (2 * S) + 96;
        p.cap = static_cast<int32_t>((cap + 31) / 32 * 32);
    } else {
        p.cap = static_cast<int32_t>(chunk / 2);
    }
    p.smem_filter = tc_smem_bytes(p.mt, p.kb, p.rb, p.kbs, p.stages, false, p.stage_half != 0);
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
    if (!make_map(&mq, Q_lp, n, kp, prec, kBlockM, 0) || !make_map(&mr, R_lp, m, kp, prec, p.rb, p.kbs))
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
    if (!make_map(&mq, Q_lp, n, kp, prec, kBlockM, 0) || !make_map(&mr, R_lp, m, kp, prec, p.rb, p.kbs))
        return cudaErrorInvalidValue;
    TcArgs a = base_args(p, n, m, error_flag);
    a.stride = 1;
    a.lists = lists;
    a.counts = counts;
    if (launches) ++*launches;
    return dispatch<false>(p, prec, mq, mr, a, st);
}

}  // namespace knn
