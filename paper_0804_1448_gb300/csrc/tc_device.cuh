// tc_device.cuh -- device code of the tensor-core stages (knn_tc.cu), shared
// with the persistent batch kernel (knn_batch.cu): the pilot / filter item
// (tc_run), the operand row preparation (prepare_row) and the per-query
// threshold (threshold_query), with the kernels that run them one launch per
// search.
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
//   filter  -- on every tile, the sign of acc says whether the reference
//              passes the query's threshold (acc >= 0); passing references are
//              appended, with their acc, to the query's list.  Half of a
//              slice's signs are collected by funnel shifts (integer pipe), the
//              other half by saturated multiplies packed with two-lane Horner
//              steps (float pipe), so the common case costs about one
//              instruction per distance, split over two pipes.  The values of
//              the few passing ones reach the dynamically indexed append
//              through shared memory: only 16-byte quarters holding a hit are
//              stored (predicated).  The key is (16-bit code of acc, index);
//              with long rows (smaller staging area) all 32 values are staged,
//              as codes packed two to a word.
// The lists then go to the finalize stage (knn_finalize.cu), which keeps the
// best c by acc, re-ranks them with exact float32 differences, and checks the
// list was neither too short nor overflowed.
//
// CTA layout: one tile of 128 queries (MMA M; one TMEM lane per query) meets
// reference tiles of 256 (MMA N = 256: one tcgen05.mma per 16- or 8-element
// K step covers the whole tile, which halves the instructions, commits and
// waits per product against N = 128):
//   warp 0        TMA producer: the query tile once, then reference tiles into
//                 a ring of shared-memory stages (128-byte swizzle), a stage
//                 being a whole tile with all its K blocks, or one K block of
//                 it when rows are long;
//   warp 1        MMA issuer: per reference tile, one tcgen05.mma per K step
//                 into one of two 256-column TMEM accumulators (all 512
//                 columns); tcgen05.commit frees the stage and publishes the tile;
//   warps 2..17   epilogue: warp w may read the TMEM lanes 32*(w%4)..+31, so
//                 thread t of warp w owns query row 32*(w%4)+t, and the four
//                 warps sharing a lane quarter take 64 columns each.  A warp
//                 loads its two 32-column slices, releases the accumulator,
//                 then works on the slices while the next tile is multiplied.
// Every mbarrier wait is bounded; on expiry the CTA raises the error flag,
// stops, waits for what it issued and frees its TMEM.
#pragma once

#include <cmath>

#include <cuda_bf16.h>

#include "knn_internal.cuh"
#include "tc_ptx.cuh"

namespace knn {
using namespace ptx;
namespace {

constexpr int kBlockM = 128;                        // queries per CTA
constexpr int kTileN = 256;                         // references per tile (MMA N)
constexpr int kAtomBytes = 128;
constexpr int kQTileBytes = kBlockM * kAtomBytes;   // one 128-byte K block of the query tile
constexpr int kRTileBytes = kTileN * kAtomBytes;    // one 128-byte K block of a reference tile
constexpr int kEpiWarps = 16;
constexpr int kEpi = 32 * kEpiWarps;                // epilogue threads
constexpr int kTcThreads = 64 + kEpi;
constexpr int kGroups = kEpiWarps / 4;              // column groups: hit lists per query and split
constexpr int kGroupCols = kTileN / kGroups;        // 64: two 32-column slices per warp
constexpr uint32_t kTmemCols = 2 * kTileN;          // two accumulators
constexpr int kMaxStages = 12;
constexpr size_t kSmemLimit = 232448;
constexpr int kAugCols = 4;
// Words per thread in the hit-staging area.  Codes: a slice's 32 values
// packed to their upper 16 bits (16 words) + pad, so that eight lanes'
// 16-byte stores fall on distinct banks.  Raw: the 32 float32 values, each
// 16-byte quarter stored only by lanes with a hit in it (few per store, so
// bank conflicts do not arise).
constexpr int kStageWords = 20;
constexpr int kStageWordsRaw = 32;

struct TcArgs {
    int64_t n, m;
    int32_t kb;           // 128-byte K blocks per operand row (row pitch = kb * 128 bytes)
    int32_t ksteps;       // 32-byte MMA K steps that carry data
    int32_t kbs;          // K blocks per stage: kb (whole tiles) or 1 (long rows)
    int32_t stages;
    int64_t chunk;        // references per split (multiple of kTileN)
    int32_t S;
    int32_t stride;       // pilot: every stride-th tile of a split
    int32_t spt;          // pilot: sampled-tile slots per split
    int32_t G;            // pilot: group maxima per query (S * spt * 8 * gps)
    int32_t gps;          // pilot: groups per 32-column slice (1, 2 or 4: groups of 32, 16, 8)
    uint32_t* gmax;       // pilot: [n][G] order-mapped maxima, 0 = no group
    uint64_t* lists;      // filter: [n][S][kGroups][cap], one list per column group
    int32_t* counts;      // filter: [n][S][kGroups] (may exceed cap: overflow)
    int32_t cap;
    int32_t append_all;   // filter: every valid reference passes
    const float* qscale;  // filter: per-query B, a power of two with |acc| < B
    int32_t* error_flag;
};

// A: the query tile, kb K blocks (resident); B: a ring of `stages` stages of
// kTileN references x kbs K blocks; hit staging (filter only); barriers.
__host__ __device__ constexpr size_t tc_smem_bytes(int kb, int kbs, int stages, bool pilot,
                                                   bool raw = false) {
    return 1024 + static_cast<size_t>(kQTileBytes) * kb +
           static_cast<size_t>(kRTileBytes) * kbs * stages +
           (pilot ? 0 : static_cast<size_t>(kEpi) * (raw ? kStageWordsRaw : kStageWords) * 4) + 512;
}

// Long rows (K-block stages): hit values are kept as a 16-bit code of acc,
// so a slice's 32 values stage in 64 bytes per thread.  With B a power of two and
// |acc| < B, acc + 3B lies in [2B, 4B), one binade, so bits 8..23 of its
// float32 pattern (the low exponent bit, constant there, and the top 15
// mantissa bits) grow with acc in steps of B 2^-14.  The list key is
// (0xffff - code, index): smaller is nearer, and the finalize reads
// 0xffff - code back as a plain number.
// The codes of two accumulator words x0, x1 (acc bits) packed into one word
// (x0's in the low half): one two-lane float32 add of 3B, then bytes 1-2 of
// each sum.
__device__ __forceinline__ uint32_t hit_code2(uint32_t x0, uint32_t x1, uint32_t off3b) {
    uint32_t y0, y1;
    asm("{\n .reg .b64 a, b;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %4};\n"
        " add.rn.f32x2 a, a, b;\n mov.b64 {%0, %1}, a;\n}"
        : "=r"(y0), "=r"(y1)
        : "r"(x0), "r"(x1), "r"(off3b));
    return __byte_perm(y0, y1, 0x6521);
}

__device__ __forceinline__ void append(uint64_t* list, int& cnt, int cap, uint32_t code, uint32_t j) {
    if (cnt < cap) list[cnt] = (static_cast<uint64_t>(0xffffu - code) << 32) | j;
    ++cnt;
}

// Raw staging: the list key of one hit from its float32 acc x, as bits 8..23
// of 3B - x (in (2B, 4B) for |x| < B, one binade): it falls with acc in steps
// of B 2^-14, like 0xffff minus the code above.
__device__ __forceinline__ void append_raw(uint64_t* list, int& cnt, int cap, float b3, float x,
                                           uint32_t j) {
    const uint32_t hi = __byte_perm(__float_as_uint(b3 - x), 0u, 0x4421);
    if (cnt < cap) list[cnt] = (static_cast<uint64_t>(hi) << 32) | j;
    ++cnt;
}

// Float-pipe pieces of the filter's pass test: fails_f(x) = 1.0 when the
// float32 x (given as bits) is negative and normal, else 0.0 (one saturated
// multiply); horner4(h, a, b) = 4 h + (a, b) on a pair of floats (one
// two-lane fused multiply-add); packed_bits(h) = the integer 2 lo + hi (at
// most 16 bits, exact in float32) read from the mantissa of 2 lo + hi + 2^23.
__device__ __forceinline__ float fails_f(uint32_t x) {
    float r;
    asm("mul.rn.ftz.sat.f32 %0, %1, 0fFE800000;" : "=f"(r) : "f"(__uint_as_float(x)));
    return r;
}
__device__ __forceinline__ uint64_t horner4(uint64_t h, float a, float b) {
    uint64_t r;
    asm("{\n .reg .b64 ab, four;\n mov.b64 ab, {%2, %3};\n mov.b64 four, {%4, %4};\n"
        " fma.rn.f32x2 %0, %1, four, ab;\n}"
        : "=l"(r) : "l"(h), "f"(a), "f"(b), "f"(4.0f));
    return r;
}
__device__ __forceinline__ uint32_t packed_bits(uint64_t h) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(h));
    return __float_as_uint(fmaf(lo, 2.f, hi + 8388608.f));
}

// Position of the highest set bit of x, in 0..31 (31 when x == 0: a valid
// staging index whose result the caller discards).
__device__ __forceinline__ uint32_t bfind31(uint32_t x) {
    uint32_t p;
    asm("bfind.u32 %0, %1;" : "=r"(p) : "r"(x));
    return p & 31u;
}

// Store v to [addr] only when bits & sel != 0 (a predicated 16-byte shared
// store; the predicate comes from the three-input logic operation itself).
__device__ __forceinline__ void st_shared_if(uint32_t bits, uint32_t sel, uint32_t addr, uint32_t v0,
                                             uint32_t v1, uint32_t v2, uint32_t v3) {
    asm volatile("{\n .reg .pred p, t;\n .reg .b32 x;\n setp.eq.u32 t, 1, 1;\n"
                 " lop3.and.b32 x|p, %0, %1, 0, 0xc0, t;\n"
                 " @p st.shared.v4.b32 [%2], {%3, %4, %5, %6};\n}"
                 :: "r"(bits), "r"(sel), "r"(addr), "r"(v0), "r"(v1), "r"(v2), "r"(v3) : "memory");
}

// MMAs of one 128-byte K block of one reference tile.  Fully unrolled over the
// four 32-byte K steps (a runtime guard skips steps past the data): issue from
// the single MMA thread must keep pace with the tensor core.  Descriptors
// advance by 32 bytes (2 in their 16-byte address field) per K step.
template <int PREC>
__device__ __forceinline__ void issue_kblock(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                             int k4, bool first, uint32_t id) {
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        if (ks < k4)
            mma<PREC>(d_tmem, a_desc + 2 * ks, b_desc + 2 * ks, id, (first && ks == 0) ? 0u : 1u);
    }
}

// KBT > 0: whole-tile stages of exactly KBT K blocks (compile-time, unrolled);
// KBT == 0: any K-block count, whole-tile or single-K-block stages.
// EPI (filter epilogue): 0 = 16-bit codes staged (long rows), 1 = raw values
// staged by quarters holding a hit, 2 = raw, every reference appended (no pilot).
// One (query tile, reference split) item of a pilot or filter pass, run by
// the whole CTA (kTcThreads threads).  smem_raw: the dynamic shared memory
// (tc_smem_bytes of this plan).  PERSIST = false: the item allocates TMEM and
// frees it at the end (one item per CTA launch); true: the caller owns the
// TMEM allocation (tmem_persist) and runs items back to back, so the item
// also invalidates its mbarriers before it returns.
template <int PREC, bool PILOT, int KBT, int EPI, bool PERSIST>
__device__ __forceinline__ void tc_run(const CUtensorMap* tmap_q, const CUtensorMap* tmap_r,
                                       const TcArgs& a, int64_t qtile, int split,
                                       unsigned char* smem_raw, uint32_t tmem_persist) {
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);

    const int KB = KBT > 0 ? KBT : a.kb, KBS = KBT > 0 ? KBT : a.kbs;
    const int NST = a.stages;
    const int SPT = KB / KBS;                   // stages per reference tile (1, or KB when KBS = 1)
    const size_t stage_bytes = static_cast<size_t>(kRTileBytes) * KBS;
    unsigned char* sA = smem;
    unsigned char* sB = sA + static_cast<size_t>(KB) * kQTileBytes;
    uint32_t* stage = reinterpret_cast<uint32_t*>(sB + NST * stage_bytes);
    constexpr bool RAW = EPI != 0;
    constexpr int kSW = RAW ? kStageWordsRaw : kStageWords;
    uint64_t* bars = reinterpret_cast<uint64_t*>(stage + (PILOT ? 0 : kEpi * kSW));
    uint64_t* full = bars;
    uint64_t* empty = bars + kMaxStages;
    uint64_t* a_full = bars + 2 * kMaxStages;
    uint64_t* t_full = a_full + 1;
    uint64_t* t_empty = t_full + 2;
    uint64_t* drain = t_empty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t q0 = qtile * kBlockM;
    const int64_t r_begin = static_cast<int64_t>(split) * a.chunk;
    const int64_t r_end = min(a.m, r_begin + a.chunk);
    const int tiles_all = static_cast<int>((r_end - r_begin + kTileN - 1) / kTileN);
    const int stride = PILOT ? a.stride : 1;
    const int nt = (tiles_all + stride - 1) / stride;   // tiles this CTA processes

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(a_full, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&t_full[b], 1);
            mbar_init(&t_empty[b], kEpiWarps);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (!PERSIST && warp == 1) tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = PERSIST ? tmem_persist : *tmem_slot;

    auto fail = [&]() {
        *abort_flag = 1;
        atomicExch(a.error_flag, 1);
    };

    if (warp == 0) {
        // -------------------------------------------------------- producer
        // one 3-D box per load: (128 bytes of K) x rows x K blocks
        if (lane == 0) {
            mbar_expect_tx(a_full, KB * kQTileBytes);
            tma_load_3d(sA, tmap_q, a_full, 0, static_cast<int>(q0), 0);
            int issued = 0;   // stage h = tile * SPT + K-block group
            for (int h = 0; h < nt * SPT; ++h) {
                const int g = h / SPT, z = (h % SPT) * KBS, s = h % NST;
                if (!mbar_wait(&empty[s], ((h / NST) & 1) ^ 1, abort_flag)) { fail(); break; }
                mbar_expect_tx(&full[s], static_cast<uint32_t>(stage_bytes));
                const int y = static_cast<int>(r_begin + static_cast<int64_t>(g) * stride * kTileN);
                tma_load_3d(sB + s * stage_bytes, tmap_r, &full[s], 0, y, z);
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
            const uint32_t id = idesc(PREC == kBF16 ? 1 : 2, kBlockM, kTileN);
            bool ok = mbar_wait(a_full, 0, abort_flag);
            if (!ok) fail();
            const uint64_t a_desc = sdesc(smem_u32(sA));
            constexpr uint32_t kQStep = kQTileBytes >> 4, kRStep = kRTileBytes >> 4;
            for (int g = 0; ok && g < nt; ++g) {
                const int buf = g & 1;
                if (!mbar_wait(&t_empty[buf], ((g >> 1) & 1) ^ 1, abort_flag)) { fail(); break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem + buf * kTileN;
                if (SPT == 1) {
                    // whole-tile stage g
                    const int s = g % NST;
                    if (!mbar_wait(&full[s], (g / NST) & 1, abort_flag)) { fail(); break; }
                    tc_fence_after();
                    const uint64_t b_desc = sdesc(smem_u32(sB + s * stage_bytes));
                    if (KBT > 0) {
#pragma unroll
                        for (int kb = 0; kb < (KBT > 0 ? KBT : 1); ++kb)
                            issue_kblock<PREC>(d_tmem, a_desc + kb * kQStep, b_desc + kb * kRStep,
                                               a.ksteps - kb * 4, kb == 0, id);
                    } else {
                        for (int kb = 0; kb < KB; ++kb)
                            issue_kblock<PREC>(d_tmem, a_desc + kb * kQStep, b_desc + kb * kRStep,
                                               a.ksteps - kb * 4, kb == 0, id);
                    }
                    tc_commit(&empty[s]);   // the stage is free once these MMAs complete
                } else {
                    // one K block per stage: tile g takes stages g*KB .. g*KB+KB-1
                    for (int kb = 0; kb < KB; ++kb) {
                        const int h = g * KB + kb, s = h % NST;
                        if (!mbar_wait(&full[s], (h / NST) & 1, abort_flag)) {
                            fail();
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        issue_kblock<PREC>(d_tmem, a_desc + kb * kQStep,
                                           sdesc(smem_u32(sB + s * stage_bytes)), a.ksteps - kb * 4,
                                           kb == 0, id);
                        tc_commit(&empty[s]);
                    }
                    if (!ok) break;
                }
                tc_commit(&t_full[buf]);
            }
            tc_commit(drain);   // arrives once every MMA issued above has completed
            mbar_wait(drain, 0, nullptr);
        }
        __syncwarp();
    } else {
        // -------------------------------------------------------- epilogue
        const int et = threadIdx.x - 64;            // 0 .. kEpi-1
        const int quarter = warp & 3;               // the TMEM lanes this warp may access
        const int cg = (warp - 2) / 4;              // column group: columns cg*64 .. +63
        const int row = quarter * 32 + lane;
        const int64_t q = q0 + row;
        const bool active = q < a.n;
        const uint32_t lane_addr = tmem + (static_cast<uint32_t>(quarter * 32) << 16);
        uint32_t* st = stage + et * kSW;
        const int gps = PILOT ? a.gps : 1;          // pilot groups per 32-column slice
        const int gpt = (kTileN / 32) * gps;        // pilot groups per tile
        uint64_t* list = nullptr;
        uint32_t* gout = nullptr;
        if (PILOT) gout = a.gmax + q * a.G + static_cast<int64_t>(split) * a.spt * gpt;
        else list = a.lists + ((q * a.S + split) * kGroups + cg) * static_cast<int64_t>(a.cap);
        const uint32_t off3b = __float_as_uint((!PILOT && active) ? 3.f * a.qscale[q] : 0.f);
        const uint32_t st_addr = smem_u32(st);
        const uint32_t all_pass = a.append_all ? 0xffffffffu : 0u;
        const uint32_t live = active ? 0xffffffffu : 0u;
        int cnt = 0;
        for (int g = 0; g < nt; ++g) {
            const int buf = g & 1;
            const bool ok = mbar_wait(&t_full[buf], (g >> 1) & 1, abort_flag);
            if (!__all_sync(0xffffffffu, ok)) { fail(); break; }
            tc_fence_after();
            const int64_t jt = r_begin + static_cast<int64_t>(g) * stride * kTileN + cg * kGroupCols;
            // valid columns of this warp's 64 (fewer only in a split's last tile)
            const int lim = static_cast<int>(min(max(r_end - jt, static_cast<int64_t>(0)),
                                                 static_cast<int64_t>(kGroupCols)));
            // both 32-column slices into registers, then release the accumulator
            uint32_t ra[32], rb[32];
            const uint32_t col0 = lane_addr + buf * kTileN + cg * kGroupCols;
            tmem_ld32u_async(col0, ra);
            tmem_ld32u_async(col0 + 32, rb);
            tmem_wait_ld2(ra, rb);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&t_empty[buf]);
            if constexpr (!PILOT && RAW) {
              if constexpr (EPI == 2) {
                // no pilot (too few references for one): every valid reference
                // is appended in column order, two keys per 16-byte store.  A
                // list holds exactly its column group's chunk / 4 columns, and
                // every slice before the last starts at a multiple of 32 keys,
                // so the stores stay inside it and 16-byte aligned.
                if (active) {
                    const float b3 = __uint_as_float(off3b);
#pragma unroll
                    for (int sl = 0; sl < 2; ++sl) {
                        const uint32_t (&r)[32] = sl ? rb : ra;
                        const int nv = min(max(lim - 32 * sl, 0), 32);
                        const uint32_t j0 = static_cast<uint32_t>(jt) + 32u * sl;
                        uint4* dst = reinterpret_cast<uint4*>(list + cnt);
#pragma unroll
                        for (int u = 0; u < 32; u += 2) {
                            if (u < nv) {
                                const uint32_t c0 = __byte_perm(
                                    __float_as_uint(b3 - __uint_as_float(r[u])), 0u, 0x4421);
                                const uint32_t c1 = __byte_perm(
                                    __float_as_uint(b3 - __uint_as_float(r[u + 1])), 0u, 0x4421);
                                if (u + 1 < nv) dst[u / 2] = make_uint4(j0 + u, c0, j0 + u + 1, c1);
                                else list[cnt + u] = (static_cast<uint64_t>(c0) << 32) | (j0 + u);
                            }
                        }
                        cnt += nv;
                    }
                }
              } else {
                // "fails" bits of both slices first (four independent chains),
                // bit 31-u for element u.  Elements 0..15: sign bits by funnel
                // shifts (integer pipe).  Elements 16..31 on the float pipe,
                // which is otherwise idle here: -acc * 2^126 saturated is 1 for a
                // negative normal acc and 0 otherwise (so -0 and negative
                // subnormals pass too: a superset of the sign test); two-lane
                // Horner steps times 4 pack them, and 2 lo + hi + 2^23 holds the
                // 16 bits in its mantissa.
                uint32_t ma = 0u, mb = 0u;
                uint64_t ha = 0ull, hb = 0ull;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    ma = __funnelshift_l(ra[u], ma, 1);
                    mb = __funnelshift_l(rb[u], mb, 1);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    ha = horner4(ha, fails_f(ra[16 + 2 * i]), fails_f(ra[17 + 2 * i]));
                    hb = horner4(hb, fails_f(rb[16 + 2 * i]), fails_f(rb[17 + 2 * i]));
                }
                // a pass is acc >= 0: bit 31-u of hits2[sl] is element u of slice sl
                uint32_t hits2[2] = {(~__byte_perm(packed_bits(ha), ma, 0x5410) | all_pass) & live,
                                     (~__byte_perm(packed_bits(hb), mb, 0x5410) | all_pass) & live};
                if (lim < kGroupCols) {   // warp-uniform: the last tile of a split
#pragma unroll
                    for (int sl = 0; sl < 2; ++sl) {
                        const int nv = min(max(lim - 32 * sl, 0), 32);
                        hits2[sl] &= nv > 0 ? (0xffffffffu << (32 - nv)) : 0u;
                    }
                }
#pragma unroll
                for (int sl = 0; sl < 2; ++sl) {
                    const uint32_t (&r)[32] = sl ? rb : ra;
                    uint32_t hits = hits2[sl];
                    // the values of the quarters holding a hit go to this
                    // thread's staging words, which the appends read back by index
#pragma unroll
                    for (int h = 0; h < 8; ++h)
                        st_shared_if(hits, 0xf0000000u >> (4 * h), st_addr + 16 * h,
                                     r[4 * h], r[4 * h + 1], r[4 * h + 2], r[4 * h + 3]);
                    const float b3 = __uint_as_float(off3b);
                    const float* stf = reinterpret_cast<const float*>(st) + 31;
                    const uint32_t jb = static_cast<uint32_t>(jt) + 32u * sl + 31u;
                    // two appends by every lane, predicated (most slices give
                    // some lane two hits), their staging loads issued together;
                    // a loop for the rare third and later
                    {
                        const uint32_t p0 = bfind31(hits);
                        const uint32_t h1 = hits & ~(1u << p0);
                        const uint32_t p1 = bfind31(h1);
                        const float x0 = stf[-static_cast<int>(p0)];
                        const float x1 = stf[-static_cast<int>(p1)];
                        if (hits != 0u) append_raw(list, cnt, a.cap, b3, x0, jb - p0);
                        if (h1 != 0u) append_raw(list, cnt, a.cap, b3, x1, jb - p1);
                        hits = h1 & ~(1u << p1);
                    }
                    while (hits) {
                        const uint32_t p = bfind31(hits);
                        hits ^= 1u << p;
                        append_raw(list, cnt, a.cap, b3, stf[-static_cast<int>(p)], jb - p);
                    }
                    // (each thread reads back only its own staging words: no
                    // warp barrier; the next tile's vote reconverges the warp)
                }
              }
            } else {
#pragma unroll
                for (int sl = 0; sl < 2; ++sl) {
                    const uint32_t (&r)[32] = sl ? rb : ra;
                    const int64_t j0 = jt + sl * 32;
                    const int64_t left = r_end - j0;
                    const int nvalid = left <= 0 ? 0 : (left >= 32 ? 32 : static_cast<int>(left));
                    if (PILOT) {
                        // halving max tree down to gps values: v[i] is then the
                        // maximum of the slice's elements u = i (mod gps), group
                        // i of the slice (valid when element i is; an absent
                        // group is written as 0, which no maximum takes)
                        float v[32];
#pragma unroll
                        for (int u = 0; u < 32; ++u)
                            v[u] = u < nvalid ? __uint_as_float(r[u]) : __int_as_float(0xff800000);
#pragma unroll
                        for (int w2 = 16; w2 > 0; w2 >>= 1)
                            if (w2 >= gps) {   // uniform
#pragma unroll
                                for (int u = 0; u < w2; ++u) v[u] = fmaxf(v[u], v[u + w2]);
                            }
                        uint32_t* go = gout + g * gpt + (cg * 2 + sl) * gps;
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (i < gps && active) go[i] = i < nvalid ? ord_f32(v[i]) : 0u;
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
                        // registers do not allow: their upper halves go through shared memory
                        if (hits) {
#pragma unroll
                            for (int h = 0; h < 4; ++h)
                                reinterpret_cast<uint4*>(st)[h] = make_uint4(
                                    hit_code2(r[8 * h + 0], r[8 * h + 1], off3b),
                                    hit_code2(r[8 * h + 2], r[8 * h + 3], off3b),
                                    hit_code2(r[8 * h + 4], r[8 * h + 5], off3b),
                                    hit_code2(r[8 * h + 6], r[8 * h + 7], off3b));
                            const uint32_t jb = static_cast<uint32_t>(j0);
                            const uint16_t* st16 = reinterpret_cast<const uint16_t*>(st);
                            do {
                                const int u = __ffs(hits) - 1;
                                hits &= hits - 1;
                                append(list, cnt, a.cap, st16[u], jb + u);
                            } while (hits);
                        }
                        __syncwarp();
                    }
                }
            }
        }
        if (!PILOT && active) a.counts[(q * a.S + split) * kGroups + cg] = cnt;
        // pilot: the group slots of tiles this split does not have (a short
        // split) hold no maximum; every slot of the row is then written, so
        // the buffer needs no clearing beforehand
        if (PILOT && active)
            for (int g = nt; g < a.spt; ++g)
                for (int i = 0; i < 2 * gps; ++i) gout[g * gpt + cg * 2 * gps + i] = 0u;
    }
    tc_fence_before();
    __syncthreads();
    if (!PERSIST && warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
    if (PERSIST && threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_inval(&full[s]);
            mbar_inval(&empty[s]);
        }
        mbar_inval(a_full);
        for (int b = 0; b < 2; ++b) {
            mbar_inval(&t_full[b]);
            mbar_inval(&t_empty[b]);
        }
        mbar_inval(drain);
    }
}

// The pilot and filter passes: one CTA per (query tile, reference split).
template <int PREC, bool PILOT, int KBT, int EPI>
__global__ void __launch_bounds__(kTcThreads, 1)
tc_kernel(const __grid_constant__ CUtensorMap tmap_q, const __grid_constant__ CUtensorMap tmap_r,
          TcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    tc_run<PREC, PILOT, KBT, EPI, false>(&tmap_q, &tmap_r, a, blockIdx.x, blockIdx.y, smem_raw, 0u);
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
__device__ __forceinline__ float get(const void* row, int t) {
    if (PREC == kBF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(row)[t]);
    return __uint_as_float(reinterpret_cast<const uint32_t*>(row)[t]);
}
// Four consecutive row elements t .. t+3 (t a multiple of 4; the row 8-byte
// aligned for bf16, 16-byte aligned for tf32) in one store.
template <int PREC>
__device__ __forceinline__ void put4(void* row, int t, float4 v) {
    if (PREC == kBF16) {
        const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
        const __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
        uint2 w;
        w.x = *reinterpret_cast<const uint32_t*>(&a);
        w.y = *reinterpret_cast<const uint32_t*>(&b);
        reinterpret_cast<uint2*>(row)[t / 4] = w;
    } else {
        uint4 w;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(w.x) : "f"(v.x));
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(w.y) : "f"(v.y));
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(w.z) : "f"(v.z));
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(w.w) : "f"(v.w));
        reinterpret_cast<uint4*>(row)[t / 4] = w;
    }
}
template <int PREC>
__device__ __forceinline__ float lowp_round(float v) {
    if (PREC == kBF16) return __bfloat162float(__float2bfloat16_rn(v));
    uint32_t b;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(b) : "f"(v));
    return __uint_as_float(b);
}

// Smallest power of two >= x (x > 0, finite).
__device__ __forceinline__ float pow2_ceil(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x007fffffu) & 0x7f800000u);
}

// The per-query B of the hit codes: |acc| = |q.r - ||r||^2/2 + t| is at most
// ||q|| ||r|| + ||r||^2/2 + |t|; the low-precision operands move that by well
// under 1%, and B carries 12.5% and a power-of-two round-up on top.
__device__ __forceinline__ float hit_scale(float nq2, float rmax2, float t) {
    const float bound = sqrtf(nq2) * sqrtf(rmax2) + 0.5f * rmax2 + fabsf(t);
    return pow2_ceil(bound * 1.125f + 1e-30f);
}

// One warp per row.  REF: [x, -nr_hi/2, -nr_lo/2, 1, 1, 0..], the float32
// squared norm, and the largest squared norm (atomic maximum on the bits of a
// non-negative float); QUERY: [x, 1, 1, 0, 0, 0..] (threshold words filled
// later) and, when qscale is given (no threshold pass follows), the hit-code
// scale for t = 0.
// Returns the row's squared float32 norm (REF, or QUERY with qscale) on every
// lane; with rmax2 and REF it also raises *rmax2 to it (one atomic per row;
// callers converting many rows per warp pass nullptr and raise it once).
template <int PREC, bool REF>
__device__ __forceinline__ float prepare_row(const float* __restrict__ X, int64_t r, int32_t d,
                                             int32_t kp, void* __restrict__ out,
                                             float* __restrict__ norms, uint32_t* __restrict__ rmax2,
                                             float* __restrict__ qscale, float* __restrict__ xcopy,
                                             int lane) {
    const float* x = X + r * d;
    const size_t elt = (PREC == kBF16) ? 2 : 4;
    void* row = static_cast<unsigned char*>(out) + static_cast<size_t>(r) * kp * elt;
    float nr = 0.f;
    if (REF || qscale) {
        for (int t = lane; t < d; t += 32) nr = fmaf(x[t], x[t], nr);
        for (int o = 16; o > 0; o >>= 1) nr += __shfl_xor_sync(0xffffffffu, nr, o);
    }
    if (lane == 0) {
        if (REF && norms) norms[r] = nr;
        if (REF && rmax2) atomicMax(rmax2, __float_as_uint(nr));
        if (!REF && qscale) qscale[r] = hit_scale(nr, __uint_as_float(*rmax2), 0.f);
    }
    const float h = -0.5f * nr;
    const float hi = lowp_round<PREC>(h);
    const float lo = lowp_round<PREC>(h - hi);
    for (int t = lane; t < kp; t += 32) {
        float v = 0.f;
        if (t < d) {
            v = x[t];
            if (!REF && xcopy) xcopy[r * d + t] = v;
        }
        else if (t == d) v = REF ? hi : 1.f;
        else if (t == d + 1) v = REF ? lo : 1.f;
        else if (t == d + 2 || t == d + 3) v = REF ? 1.f : 0.f;
        put<PREC>(row, t, v);
    }
    return nr;
}

constexpr int kPrepRowsPerWarp = 4;

// kPrepRowsPerWarp rows per warp.  Rows of up to 128 coordinates: every
// lane's loads of all the rows are issued before any is used (over the
// CPU-GPU link, when X is in host memory, the latency is long), then each row
// as prepare_row does it, with the same arithmetic in the same order.  Longer
// rows: prepare_row, one row after another.
template <int PREC, bool REF>
__global__ void prepare_kernel(const float* __restrict__ X, int64_t rows, int32_t d, int32_t kp,
                               void* __restrict__ out, float* __restrict__ norms,
                               uint32_t* __restrict__ rmax2, float* __restrict__ qscale,
                               float* __restrict__ xcopy) {
    constexpr int RW = kPrepRowsPerWarp;
    const int lane = threadIdx.x % 32;
    const int64_t r0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / 32 * RW;
    if (r0 >= rows) return;
    if (d > 128) {
        for (int u = 0; u < RW && r0 + u < rows; ++u)
            prepare_row<PREC, REF>(X, r0 + u, d, kp, out, norms, rmax2, qscale, xcopy, lane);
        return;
    }
    float xv[RW][4];
#pragma unroll
    for (int u = 0; u < RW; ++u)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int t = lane + 32 * j;
            xv[u][j] = (r0 + u < rows && t < d) ? X[(r0 + u) * d + t] : 0.f;
        }
    float nr[RW];
#pragma unroll
    for (int u = 0; u < RW; ++u) {
        nr[u] = 0.f;
        if (REF || qscale) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (lane + 32 * j < d) nr[u] = fmaf(xv[u][j], xv[u][j], nr[u]);
        }
    }
    if (REF || qscale) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int u = 0; u < RW; ++u) nr[u] += __shfl_xor_sync(0xffffffffu, nr[u], o);
    }
    const size_t elt = (PREC == kBF16) ? 2 : 4;
#pragma unroll
    for (int u = 0; u < RW; ++u) {
        const int64_t r = r0 + u;
        if (r >= rows) break;
        if (lane == 0) {
            if (REF && norms) norms[r] = nr[u];
            if (REF && rmax2) atomicMax(rmax2, __float_as_uint(nr[u]));
            if (!REF && qscale) qscale[r] = hit_scale(nr[u], __uint_as_float(*rmax2), 0.f);
        }
        const float h = -0.5f * nr[u];
        const float hi = lowp_round<PREC>(h);
        const float lo = lowp_round<PREC>(h - hi);
        void* row = static_cast<unsigned char*>(out) + static_cast<size_t>(r) * kp * elt;
#pragma unroll
        for (int j = 0; j < 8; ++j) {   // kp <= 256 when d <= 128
            const int t = lane + 32 * j;
            if (t >= kp) break;
            float v = 0.f;
            if (t < d) {
                v = xv[u][j < 4 ? j : 0];
                if (!REF && xcopy) xcopy[r * d + t] = v;
            }
            else if (t == d) v = REF ? hi : 1.f;
            else if (t == d + 1) v = REF ? lo : 1.f;
            else if (t == d + 2 || t == d + 3) v = REF ? 1.f : 0.f;
            put<PREC>(row, t, v);
        }
    }
}

// One warp per query: the cprime-th largest group maximum of the pilot becomes
// the query's threshold, written into its threshold words with a margin that
// covers the rounding difference between the pilot and filter products.  The
// maxima (order-mapped, 0 = no group) sit in registers, VPL per lane; the
// order statistic is found bit by bit from the top (is the count of values
// >= prefix|bit at least cprime?) down to bit 8.  Stopping there leaves a
// value at most 2^8 order steps (2^-15 relative) below the exact one: a
// slightly lower threshold, so never fewer passing references.
template <int PREC, int VPL>
__device__ __forceinline__ void threshold_query(const uint32_t* __restrict__ gmax, int64_t q,
                                                int32_t G, int32_t cprime, int32_t d, int32_t kp,
                                                void* __restrict__ Q_lp,
                                                const uint32_t* __restrict__ rmax2,
                                                float* __restrict__ qscale, int lane) {
    const uint32_t* src = gmax + q * G;
    // squared norm of the (low-precision) query row, for the hit-code scale
    const size_t elt = (PREC == kBF16) ? 2 : 4;
    void* row = static_cast<unsigned char*>(Q_lp) + static_cast<size_t>(q) * kp * elt;
    float nq2 = 0.f;
    for (int t = lane; t < d; t += 32) {
        const float x = get<PREC>(row, t);
        nq2 = fmaf(x, x, nq2);
    }
    for (int o = 16; o > 0; o >>= 1) nq2 += __shfl_xor_sync(0xffffffffu, nq2, o);
    uint32_t v[VPL];
    uint32_t least = 0xffffffffu, most = 0u;
    int nvalid = 0;
#pragma unroll
    for (int i = 0; i < VPL; ++i) {
        const int g = i * 32 + lane;
        v[i] = (g < G) ? src[g] : 0u;
        if (v[i] != 0u) {
            least = min(least, v[i]);
            most = max(most, v[i]);
            ++nvalid;
        }
    }
    least = __reduce_min_sync(0xffffffffu, least);
    most = __reduce_max_sync(0xffffffffu, most);
    nvalid = __reduce_add_sync(0xffffffffu, nvalid);
    // every group maximum, hence the answer, shares the bits above the highest
    // bit in which the largest and the smallest differ: start from them
    const uint32_t diff = most ^ least;
    const int top = 31 - __clz(diff);                 // -1 when all are equal
    uint32_t prefix = top < 0 ? most : (top >= 31 ? 0u : (most & ~((2u << top) - 1u)));
    for (int b = top; b >= 8; --b) {
        const uint32_t cand = prefix | (1u << b);
        int c = 0;
#pragma unroll
        for (int i = 0; i < VPL; ++i) c += (v[i] >= cand) ? 1 : 0;
        if (__reduce_add_sync(0xffffffffu, c) >= cprime) prefix = cand;
    }
    const uint32_t best = nvalid >= cprime ? prefix : least;   // fewer than cprime groups: the weakest
    const float t_acc = unord_f32(best);
    const float tcol = -t_acc + 1e-3f * (1.f + fabsf(t_acc));
    const float hi = lowp_round<PREC>(tcol);
    const float lo = lowp_round<PREC>(tcol - hi);
    if (lane == 0) {
        put<PREC>(row, d + 2, hi);
        put<PREC>(row, d + 3, lo);
        qscale[q] = hit_scale(nq2, __uint_as_float(*rmax2), tcol);
    }
}

template <int PREC, int VPL>
__global__ void threshold_kernel(const uint32_t* __restrict__ gmax, int64_t n, int32_t G,
                                 int32_t cprime, int32_t d, int32_t kp, void* __restrict__ Q_lp,
                                 const uint32_t* __restrict__ rmax2, float* __restrict__ qscale) {
    const int64_t q = static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32;
    if (q >= n) return;
    threshold_query<PREC, VPL>(gmax, q, G, cprime, d, kp, Q_lp, rmax2, qscale, threadIdx.x % 32);
}

}  // namespace

// rows x kp operand copy seen by TMA as 3-D boxes of box_rows rows (all K
// blocks when box_kb = 0); false if the driver entry point is missing.
bool tc_make_map(CUtensorMap* map, const void* base, int64_t rows, int kp, int prec, int box_rows,
                 int box_kb);

}  // namespace knn
