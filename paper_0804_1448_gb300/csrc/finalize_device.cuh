// finalize_device.cuh -- device code of the finalize and exact-fallback
// stages (knn_finalize.cu), shared with the persistent batch kernel
// (knn_batch.cu): the per-query finalize (finalize_query, one warp), the
// per-query fallback (fb_query and its pieces, one CTA of NT threads), and the
// kernels that run them one launch per search.
//
// finalize (one warp per query):
//   1. candidates: the S*c keys of the select stage, or the tensor-core hit
//      lists cut to (at least) the best c by their low-precision keys; then the
//      exact float32 distance of every candidate from coordinate differences
//      (the select stages rank low-precision scores or, for the Euclidean
//      CUDA-core select, lower bounds from the expanded form): the "re-rank";
//   2. ascending prefix by (distance, index) -- step 2 of the brute-force
//      algorithm of Sec. 2.1, restricted to the candidates: the first k, and
//      the run of near-equal distances that crosses position k-1;
//   3. near-tie re-check: consecutive prefix entries whose float32 distances
//      are within twice the float32 rounding bound may be out of exact order.
//      Every such run is re-evaluated as a float-float sum (error far below the
//      float32 window); entries whose float-float values are still within that
//      sum's own error bound of a run neighbour are recomputed in float64 with
//      the oracle's arithmetic (widen, subtract, square or abs, add,
//      coordinate 0 first, no fused multiply-add).  Each run is then ordered by
//      (refined distance, index);
//   4. completeness check (float32 candidates only): the references that are
//      not candidates have float32 distances >= the largest key kept by their
//      split; if that bound, lowered by the rounding bound, does not exceed the
//      k-th distance, a non-candidate could still belong to the answer and the
//      query is queued for the fallback instead of being written;
//   5. the k outputs (Euclidean: square root of the squared distance).
//
// fallback (one CTA per queued query): float32 distances to all m references,
// the k-th by radix selection, float64 distances for every reference that
// could still be in the answer, an exact radix selection, a sort, the outputs.
#pragma once

#include "knn_internal.cuh"

namespace knn {
namespace {

constexpr int kMaxPool = 4096;
constexpr int kRegPool = 128;            // pools up to 4 x 32 keys: prefix selection in registers
constexpr int kSortedStripe = 48;        // larger pools up to 48 x 32 keys: per-lane sorted stripes
constexpr int kRegHits = 16;             // hit-list entries per lane held in registers
constexpr int kStage = 32 * kRegHits;    // hit lists up to this length are staged in shared memory
constexpr int kBins = 64;
constexpr int kFinThreads = 256;

// Relative rounding bound of the float32 distance (squared Euclidean or
// Manhattan) accumulated over d coordinates with one rounding per difference
// and one per accumulation step: |d32 - d| <= (d + 2) u d, u = 2^-24.
// A safety factor of 2 covers the second-order terms.
__host__ __device__ inline double f32_rel_bound(int d) {
    return 2.0 * (d + 2) * 5.9604644775390625e-8;
}

// Relative error bound of the float-float distance below: the low word stays
// below 4(d+2) 2^-24 of the sum and is rounded at most twice per term, so the
// sum is within (d+2)^2 2^-45 of the exact one; the oracle's float64 sum is
// within (d+2) 2^-53 of it.
__host__ __device__ inline double ff_rel_bound(int d) {
    const double e = static_cast<double>(d + 2);
    return e * e * 2.8421709430404007e-14 + e * 1.1102230246251565e-16;
}

// One coordinate's contribution: squared (L2), absolute value added (L1) or
// maximum of absolute values (L-infinity, Chebyshev).
template <int METRIC>
__device__ __forceinline__ float acc_f32(float acc, float diff) {
    if (METRIC == kL2) return fmaf(diff, diff, acc);
    if (METRIC == kL1) return acc + fabsf(diff);
    return fmaxf(acc, fabsf(diff));
}
template <int METRIC>
__device__ __forceinline__ float combine_f32(float a, float b) {
    return METRIC == kLinf ? fmaxf(a, b) : a + b;
}

template <int METRIC>
__device__ __forceinline__ float dist_f32(const float* q, const float* __restrict__ r, int d) {
    float acc = 0.f;
    if ((d & 3) == 0 && ((reinterpret_cast<uintptr_t>(r) | reinterpret_cast<uintptr_t>(q)) & 15) == 0) {
        // 16-byte aligned rows: vector loads, same order of operations
        const float4* r4 = reinterpret_cast<const float4*>(r);
        const float4* q4 = reinterpret_cast<const float4*>(q);
        for (int t = 0; t < d / 4; ++t) {
            const float4 x = __ldg(r4 + t);
            const float4 y = q4[t];
            acc = acc_f32<METRIC>(acc, y.x - x.x);
            acc = acc_f32<METRIC>(acc, y.y - x.y);
            acc = acc_f32<METRIC>(acc, y.z - x.z);
            acc = acc_f32<METRIC>(acc, y.w - x.w);
        }
        return acc;
    }
    for (int t = 0; t < d; ++t) acc = acc_f32<METRIC>(acc, q[t] - __ldg(r + t));
    return acc;
}

// The oracle's float64 arithmetic, operation for operation.
template <int METRIC>
__device__ __forceinline__ double dist_f64(const float* q, const float* __restrict__ r, int d) {
    double acc = 0.0;
    for (int t = 0; t < d; ++t) {
        const double diff = __dsub_rn(static_cast<double>(q[t]), static_cast<double>(__ldg(r + t)));
        if (METRIC == kL2) acc = __dadd_rn(acc, __dmul_rn(diff, diff));
        else if (METRIC == kL1) acc = __dadd_rn(acc, fabs(diff));
        else acc = fmax(acc, fabs(diff));
    }
    return acc;
}

// ---- float-float arithmetic (round to nearest, no contraction) -----------

// s + e == a + b exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (H, Lo) += the term of coordinate pair (x, y): (x - y)^2 or |x - y|.
// x - y = s + e exactly; s^2 = p + (s^2 - p) exactly with one fused
// multiply-add; the 2se cross term joins the low word, e^2 (<= 2^-48 s^2) is
// dropped.
template <int METRIC>
__device__ __forceinline__ void ff_term(float& H, float& Lo, float x, float y) {
    float s, e;
    two_sum(x, -y, s, e);
    float p, t;
    if (METRIC == kL2) {
        p = __fmul_rn(s, s);
        t = fmaf(__fadd_rn(s, s), e, fmaf(s, s, -p));
    } else {
        const bool neg = s < 0.f;   // s == 0 only when x == y, and then e == 0
        p = neg ? -s : s;
        t = neg ? -e : e;
    }
    if (METRIC == kLinf) {
        // the exact |x - y| = p + t; keep the larger pair (both normalised)
        if (p > H || (p == H && t > Lo)) { H = p; Lo = t; }
        return;
    }
    float hs, he;
    two_sum(H, p, hs, he);
    H = hs;
    Lo = __fadd_rn(Lo, __fadd_rn(t, he));
}

template <int METRIC = kL2>
__device__ __forceinline__ void ff_combine(float& H, float& Lo, float H2, float Lo2) {
    if (METRIC == kLinf) {
        if (H2 > H || (H2 == H && Lo2 > Lo)) { H = H2; Lo = Lo2; }
        return;
    }
    float s, e;
    two_sum(H, H2, s, e);
    H = s;
    Lo = __fadd_rn(Lo, __fadd_rn(Lo2, e));
}

// A float-float value, renormalized (|lo| <= half an ulp of hi), packed as
// (bits(hi) << 32) | bits(lo).  Distances are >= 0, so hi orders by its bits
// and pairs order lexicographically (hi, then lo as a float).
__device__ __forceinline__ uint64_t ff_pack(float H, float Lo) {
    const float hi = __fadd_rn(H, Lo);
    const float lo = __fsub_rn(Lo, __fsub_rn(hi, H));
    return (static_cast<uint64_t>(__float_as_uint(hi)) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ float ff_hi(uint64_t v) { return __uint_as_float(static_cast<uint32_t>(v >> 32)); }
__device__ __forceinline__ float ff_lo(uint64_t v) { return __uint_as_float(static_cast<uint32_t>(v)); }
__device__ __forceinline__ bool ff_less(uint64_t a, uint64_t b) {
    const uint32_t ah = static_cast<uint32_t>(a >> 32), bh = static_cast<uint32_t>(b >> 32);
    return ah < bh || (ah == bh && ff_lo(a) < ff_lo(b));
}

__device__ __forceinline__ uint64_t dbits(double x) {
    return static_cast<uint64_t>(__double_as_longlong(x));
}
__device__ __forceinline__ double bitsd(uint64_t b) {
    return __longlong_as_double(static_cast<long long>(b));
}

// True when b (>= a) is within the float32 rounding of a, i.e. the exact
// order of the two can differ from their float32 order.  Evaluated in float:
// b - a is exact when a <= b <= 2a (and only larger otherwise), and relf
// carries a 1% margin over 2 * rel for the rounding of relf * b.
__device__ __forceinline__ bool near_tie(float a, float b, float relf) {
    return b - a <= relf * b + 1e-37f;
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Per-warp shared scratch of the finalize kernel.
struct WarpScratch {
    uint64_t* keys;    // [P] candidates: reference index, then exact float32 key; kEmptyKey = none
    uint64_t* stage;   // [kStage] the query's hit-list entries (shares space with sorted..rlist)
    uint64_t* sorted;  // [L] ascending prefix
    uint64_t* d64;     // [L] refined distance (float64 bits) of re-checked prefix entries
    int32_t* perm;     // [L] output position -> prefix position inside re-checked runs
    int32_t* runs;     // [L] run start of a re-checked prefix entry, -1 otherwise
    int32_t* rend;     // [L] run end (inclusive)
    int32_t* rlist;    // [L] prefix positions of the re-checked entries
    uint64_t* smax;    // [S] largest select-stage key per split
    int32_t* hist;     // [kBins + 4]
    float* qrow;       // [d + 4], 16-byte aligned
};

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~static_cast<size_t>(15); }

// Layout (every array 16-byte aligned): keys [P] u64; then either the hit
// staging area [kStage] u64 or, once it is consumed, sorted, d64 [L] u64 and
// perm, runs, rend, rlist [L] i32; smax [S] u64; hist [kBins+4] i32; qrow
// [d+4] f32.  L bounds the sorted prefix (the first k and the near-tie run
// that crosses position k-1).
__host__ __device__ inline size_t prefix_bytes(int L) {
    return align16(static_cast<size_t>(L) * 8) * 2 + align16(static_cast<size_t>(L) * 4) * 4;
}
__host__ __device__ inline size_t warp_scratch_bytes(int P, int L, int S, int d, int stage_entries) {
    const size_t u = prefix_bytes(L);
    const size_t st = static_cast<size_t>(stage_entries) * 8;
    return align16(static_cast<size_t>(P) * 8) + (u > st ? u : st) +
           align16(static_cast<size_t>(S) * 8) + align16((kBins + 4) * 4) +
           align16((static_cast<size_t>(d) + 4) * 4);
}

__host__ __device__ inline int prefix_cap(int P, int k) { return P < k + 64 ? P : k + 64; }

__device__ __forceinline__ WarpScratch carve(unsigned char* base, int P, int L, int S, int stage_entries) {
    WarpScratch w;
    size_t o = 0;
    w.keys = reinterpret_cast<uint64_t*>(base + o);   o += align16(static_cast<size_t>(P) * 8);
    const size_t u0 = o;
    w.stage = reinterpret_cast<uint64_t*>(base + o);
    w.sorted = reinterpret_cast<uint64_t*>(base + o); o += align16(static_cast<size_t>(L) * 8);
    w.d64 = reinterpret_cast<uint64_t*>(base + o);    o += align16(static_cast<size_t>(L) * 8);
    w.perm = reinterpret_cast<int32_t*>(base + o);    o += align16(static_cast<size_t>(L) * 4);
    w.runs = reinterpret_cast<int32_t*>(base + o);    o += align16(static_cast<size_t>(L) * 4);
    w.rend = reinterpret_cast<int32_t*>(base + o);    o += align16(static_cast<size_t>(L) * 4);
    w.rlist = reinterpret_cast<int32_t*>(base + o);   o += align16(static_cast<size_t>(L) * 4);
    const size_t st = static_cast<size_t>(stage_entries) * 8;
    if (o < u0 + st) o = u0 + st;
    w.smax = reinterpret_cast<uint64_t*>(base + o);   o += align16(static_cast<size_t>(S) * 8);
    w.hist = reinterpret_cast<int32_t*>(base + o);    o += align16((kBins + 4) * 4);
    w.qrow = reinterpret_cast<float*>(base + o);
    return w;
}

// Two-lane float32 arithmetic on pairs of consecutive coordinates held as
// 64-bit registers (as loaded, 16 bytes = two pairs): acc + (a - b)^2 per lane
// (one two-lane subtraction, one two-lane fused multiply-add), and the sum of
// a pair.
__device__ __forceinline__ uint64_t f2_sqdiff_acc(uint64_t a, uint64_t b, uint64_t acc) {
    uint64_t r;
    asm("{\n .reg .b64 t;\n sub.rn.f32x2 t, %1, %2;\n fma.rn.f32x2 %0, t, t, %3;\n}"
        : "=l"(r) : "l"(a), "l"(b), "l"(acc));
    return r;
}
__device__ __forceinline__ float pair_lo(uint64_t v) { return __uint_as_float(static_cast<uint32_t>(v)); }
__device__ __forceinline__ float pair_hi(uint64_t v) { return __uint_as_float(static_cast<uint32_t>(v >> 32)); }
__device__ __forceinline__ float f2_sum(uint64_t v) { return pair_lo(v) + pair_hi(v); }

// Replace raw reference indices keys[0..cnt) (kEmptyKey = none) by exact
// float32 keys.  NV > 0 (d % 4 == 0, d <= 128, NV = ceil(d/32)): eight lanes
// share one candidate, lane `sub` taking float4 number sub + 8v (v < NV) of
// the row, so one warp instruction reads four rows in 128-byte segments;
// every lane issues the loads of G candidates before using any of them, and
// three shuffles finish each sum.  Euclidean: the lane's coordinates go
// through two-lane float32 instructions, as four partial sums (x, y, z, w
// columns) added at the end; the rounding bound of the float32 distance holds
// for any order of the additions.  NV == 0: one lane per candidate.
template <int METRIC, int NV>
__device__ void exact_keys(uint64_t* keys, int cnt, const float* __restrict__ R, int d,
                           const float* qrow, int lane) {
    if constexpr (NV > 0) {
        constexpr int G = NV >= 3 ? 2 : (NV == 2 ? 3 : 4);
        const int g = lane >> 3, sub = lane & 7, d4 = d >> 2;
        const ulonglong2* q4 = reinterpret_cast<const ulonglong2*>(qrow);
        for (int e0 = 0; e0 < cnt; e0 += 4 * G) {
            uint64_t raw[G];
            ulonglong2 x[G][NV];   // four coordinates as two pairs
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const int e = e0 + 4 * u + g;
                raw[u] = (e < cnt) ? keys[e] : kEmptyKey;
                const ulonglong2* row = reinterpret_cast<const ulonglong2*>(
                    R + static_cast<int64_t>(raw[u] == kEmptyKey ? 0 : raw[u]) * d);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const int t = sub + 8 * v;
                    x[u][v] = (raw[u] != kEmptyKey && t < d4) ? __ldg(row + t) : make_ulonglong2(0ull, 0ull);
                }
            }
            float acc[G];
            if constexpr (METRIC == kL2) {
                uint64_t s01[G], s23[G];
#pragma unroll
                for (int u = 0; u < G; ++u) s01[u] = s23[u] = 0ull;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const int t = sub + 8 * v;
                    if (t < d4) {
                        const ulonglong2 y = q4[t];
#pragma unroll
                        for (int u = 0; u < G; ++u) {
                            s01[u] = f2_sqdiff_acc(y.x, x[u][v].x, s01[u]);
                            s23[u] = f2_sqdiff_acc(y.y, x[u][v].y, s23[u]);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < G; ++u) acc[u] = f2_sum(s01[u]) + f2_sum(s23[u]);
            } else {
#pragma unroll
                for (int u = 0; u < G; ++u) acc[u] = 0.f;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const int t = sub + 8 * v;
                    if (t < d4) {
                        const ulonglong2 y = q4[t];
#pragma unroll
                        for (int u = 0; u < G; ++u) {
                            const ulonglong2 r = x[u][v];
                            acc[u] = acc_f32<METRIC>(acc[u], pair_lo(y.x) - pair_lo(r.x));
                            acc[u] = acc_f32<METRIC>(acc[u], pair_hi(y.x) - pair_hi(r.x));
                            acc[u] = acc_f32<METRIC>(acc[u], pair_lo(y.y) - pair_lo(r.y));
                            acc[u] = acc_f32<METRIC>(acc[u], pair_hi(y.y) - pair_hi(r.y));
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < G; ++u) {
                float v = acc[u];
                v = combine_f32<METRIC>(v, __shfl_xor_sync(0xffffffffu, v, 4));
                v = combine_f32<METRIC>(v, __shfl_xor_sync(0xffffffffu, v, 2));
                v = combine_f32<METRIC>(v, __shfl_xor_sync(0xffffffffu, v, 1));
                const int e = e0 + 4 * u + g;
                if (sub == 0 && raw[u] != kEmptyKey)
                    keys[e] = make_key(v, static_cast<uint32_t>(raw[u]));
            }
        }
    } else {
        for (int e = lane; e < cnt; e += 32) {
            const uint64_t raw = keys[e];
            if (raw != kEmptyKey)
                keys[e] = make_key(dist_f32<METRIC>(qrow, R + static_cast<int64_t>(raw) * d, d),
                                   static_cast<uint32_t>(raw));
        }
    }
    __syncwarp();
}

// Float-float distances of the prefix entries listed in rlist[0..nr), as
// float64 bits in d64[position].  Same lane layout as exact_keys.
template <int METRIC, int NV>
__device__ void refine_ff(const WarpScratch& w, int nr, const float* __restrict__ R, int d, int lane) {
    if constexpr (NV > 0) {
        const int g = lane >> 3, sub = lane & 7, d4 = d >> 2;
        const float4* q4 = reinterpret_cast<const float4*>(w.qrow);
        for (int e0 = 0; e0 < nr; e0 += 4) {
            const int e = e0 + g;
            const int p = (e < nr) ? w.rlist[e] : -1;
            float H = 0.f, Lo = 0.f;
            if (p >= 0) {
                const float4* row = reinterpret_cast<const float4*>(
                    R + static_cast<int64_t>(key_idx(w.sorted[p])) * d);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const int t = sub + 8 * v;
                    if (t < d4) {
                        const float4 r = __ldg(row + t);
                        const float4 y = q4[t];
                        ff_term<METRIC>(H, Lo, y.x, r.x);
                        ff_term<METRIC>(H, Lo, y.y, r.y);
                        ff_term<METRIC>(H, Lo, y.z, r.z);
                        ff_term<METRIC>(H, Lo, y.w, r.w);
                    }
                }
            }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                const float H2 = __shfl_xor_sync(0xffffffffu, H, o);
                const float L2 = __shfl_xor_sync(0xffffffffu, Lo, o);
                ff_combine<METRIC>(H, Lo, H2, L2);
            }
            if (sub == 0 && p >= 0) w.d64[p] = ff_pack(H, Lo);
        }
    } else {
        for (int e = lane; e < nr; e += 32) {
            const int p = w.rlist[e];
            const float* r = R + static_cast<int64_t>(key_idx(w.sorted[p])) * d;
            float H = 0.f, Lo = 0.f;
            for (int t = 0; t < d; ++t) ff_term<METRIC>(H, Lo, w.qrow[t], __ldg(r + t));
            w.d64[p] = ff_pack(H, Lo);
        }
    }
    __syncwarp();
}

// Candidate-set front end: exact float32 keys of the S*c entries of query q,
// and the largest select-stage key of every split.
template <int METRIC, int NV>
__device__ void gather_cand(const FinalizeArgs& a, int64_t q, WarpScratch& w, int lane) {
    const CandidateSet& cs = a.cand;
    const int Sc = cs.S * cs.c;
    const uint64_t* src = cs.keys + q * static_cast<int64_t>(Sc);
    for (int e = lane; e < Sc; e += 32) {
        const uint64_t key = src[e];
        uint64_t raw = kEmptyKey;
        if (key != kEmptyKey) {
            raw = key_idx(key);
            atomicMax(reinterpret_cast<unsigned long long*>(&w.smax[e / cs.c]),
                      static_cast<unsigned long long>(key));
        }
        w.keys[e] = raw;
    }
    __syncwarp();
    exact_keys<METRIC, NV>(w.keys, Sc, a.R, a.d, w.qrow, lane);
}

// The score of a hit-list key: its high word, a code in [0, 0xffff] that
// falls linearly with the low-precision score, as a float (exact: the code
// sits in the mantissa of 2^23 + code).
__device__ __forceinline__ float hit_val(uint32_t hi) {
    return __uint_as_float(0x4B000000u | hi) - 8388608.f;
}

// First-level histogram over [vmin, vmax]: inv = (kBins - 0.51) / (vmax - vmin),
// so (v - lo) * inv lies in [0, kBins - 0.51] and one fused multiply-add onto
// 1.5 * 2^23 rounds it to an integer held in the low mantissa bits.
struct FastBin {
    float lo, inv;
    __device__ int bin(float v) const {
        return __float_as_int(fmaf(v - lo, inv, 12582912.f)) & (kBins - 1);
    }
};

// Histogram over [lo, lo + kBins/inv), values outside clamped to the ends.
struct Binning {
    float lo, inv;
    __device__ int bin(float v) const {
        const float x = (v - lo) * inv;
        return x <= 0.f ? 0 : (x >= kBins - 1 ? kBins - 1 : static_cast<int>(x));
    }
};

// Smallest bin whose cumulative count reaches `need`, and the cumulative
// count before it.  Two bins per lane.
__device__ void cut_bin(const int32_t* hist, int need, int lane, int* bin, int* before) {
    const int h0 = hist[2 * lane], h1 = hist[2 * lane + 1];
    int incl = h0 + h1;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int excl = incl - h0 - h1;
    int mine = kBins, mb = 0;
    if (excl + h0 >= need) { mine = 2 * lane; mb = excl; }
    else if (incl >= need) { mine = 2 * lane + 1; mb = excl + h0; }
    int best = mine;
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    const unsigned own = __ballot_sync(0xffffffffu, mine == best && best < kBins);
    *bin = best;
    *before = own ? __shfl_sync(0xffffffffu, mb, __ffs(own) - 1) : 0;
}

// Sizes of the query's hit lists: total entries and whether one overflowed.
__device__ __forceinline__ void hit_totals(const FinalizeArgs& a, int64_t q, int lane, int* total,
                                           int* over) {
    const HitLists& hl = a.hits;
    const int32_t* cnts = hl.counts + q * static_cast<int64_t>(hl.S);
    int t = 0, o = 0;
    for (int s = lane; s < hl.S; s += 32) {
        const int cs = cnts[s];
        o |= cs > hl.cap;
        t += min(cs, hl.cap);
    }
    *total = __reduce_add_sync(0xffffffffu, t);
    *over = __reduce_or_sync(0xffffffffu, o);
}

// Hit-list front end: keep the listed references whose low-precision key is
// among the best c, cutting at a histogram bin (refined once), so at least c
// and usually a few more are kept; their exact float32 keys go to w.keys.
// Returns the number kept, or -1 (list shorter than c), -2 (overflowed),
// -3 (the cut kept more than P) to send the query to the exact fallback.
// Lists of up to kStage entries are copied once into shared memory (8-byte
// asynchronous copies, all in flight together) and their keys held in
// registers (MODE 1).  Lists that fit the warp's whole key and staging area
// (keys[P] and the staging words are adjacent) are copied there and every
// pass reads shared memory; the kept indices are compacted in place, each
// written at or before the position it was read from (MODE 2).  Longer ones
// are re-read from global memory at every pass (MODE 0).
template <int METRIC, int NV, int MODE>
__device__ int gather_hits_impl(const FinalizeArgs& a, int64_t q, int P, WarpScratch& w, int lane,
                                int total) {
    constexpr bool STAGED = MODE != 0;
    const HitLists& hl = a.hits;
    const int S = hl.S, cap = hl.cap, c = hl.c;
    const uint64_t* base = hl.keys + q * static_cast<int64_t>(S) * cap;
    const int32_t* cnts = hl.counts + q * static_cast<int64_t>(S);
    // every listed key straight from global memory (MODE 0): many short lists
    // (many reference splits) are walked one list per lane, all lanes at once;
    // a few long lists one list at a time, its entries over the lanes
    auto visit_global = [&](auto&& g) {
        if (S >= 16) {
            for (int s = lane; s < S; s += 32) {
                const int cs = min(cnts[s], cap);
                const uint64_t* sp = base + static_cast<int64_t>(s) * cap;
                for (int e = 0; e < cs; ++e) g(sp[e]);
            }
        } else {
            for (int s = 0; s < S; ++s) {
                const int cs = min(cnts[s], cap);
                const uint64_t* sp = base + static_cast<int64_t>(s) * cap;
                for (int e = lane; e < cs; e += 32) g(sp[e]);
            }
        }
    };
    uint32_t hv[MODE == 1 ? kRegHits : 1];   // high words of the staged keys (order of the score)
    uint64_t* const dst = MODE == 2 ? w.keys : w.stage;
    if constexpr (STAGED) {
        int o = 0;
        for (int s0 = 0; s0 < S; s0 += 32) {
            const int mine = (s0 + lane < S) ? min(cnts[s0 + lane], cap) : 0;
            int incl = mine;
            for (int sh = 1; sh < 32; sh <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, sh);
                if (lane >= sh) incl += v;
            }
            const int ns = min(32, S - s0);
            for (int s = 0; s < ns; ++s) {
                const int cs = __shfl_sync(0xffffffffu, mine, s);
                const int os = o + __shfl_sync(0xffffffffu, incl, s) - cs;
                const uint64_t* sp = base + static_cast<int64_t>(s0 + s) * cap;
                for (int x = lane; x < cs; x += 32) cp_async8(dst + os + x, sp + x);
            }
            o += __shfl_sync(0xffffffffu, incl, 31);
        }
        cp_async_wait_all();
        __syncwarp();
        if constexpr (MODE == 1) {
#pragma unroll
            for (int i = 0; i < kRegHits; ++i) {
                const int e = i * 32 + lane;
                hv[i] = (e < total) ? static_cast<uint32_t>(w.stage[e] >> 32) : 0u;
            }
        }
    }
    float vmin = __int_as_float(0x7f800000), vmax = -vmin;
    // visit every entry: f(score) for the staged registers, or f(key) re-read
    auto for_each = [&](auto&& f) {
        if constexpr (MODE == 1) {
#pragma unroll
            for (int i = 0; i < kRegHits; ++i)
                if (i * 32 + lane < total) f(hit_val(hv[i]));
        } else if constexpr (MODE == 2) {
            for (int e = lane; e < total; e += 32) f(hit_val(static_cast<uint32_t>(w.keys[e] >> 32)));
        } else {
            visit_global([&](uint64_t key) { f(hit_val(static_cast<uint32_t>(key >> 32))); });
        }
    };
    for_each([&](float v) {
        vmin = fminf(vmin, v);
        vmax = fmaxf(vmax, v);
    });
    for (int o = 16; o > 0; o >>= 1) {
        vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
        vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    }
    const float range = vmax - vmin;
    FastBin b1{vmin, range > 1e-30f ? (kBins - 0.51f) / range : 0.f};
    int cut1 = kBins - 1, cut2 = kBins - 1;
    Binning b2{0.f, 0.f};
    if (total > c) {
        for (int b = lane; b < kBins; b += 32) w.hist[b] = 0;
        __syncwarp();
        for_each([&](float v) { atomicAdd(&w.hist[b1.bin(v)], 1); });
        __syncwarp();
        int before;
        cut_bin(w.hist, c, lane, &cut1, &before);
        const int in_bin = w.hist[cut1];
        __syncwarp();
        if (before + in_bin > P && b1.inv > 0.f) {   // refine the cut bin once
            b2.lo = vmin + (cut1 - 0.5f) / b1.inv;
            b2.inv = b1.inv * kBins;
            for (int b = lane; b < kBins; b += 32) w.hist[b] = 0;
            __syncwarp();
            for_each([&](float v) {
                if (b1.bin(v) == cut1) atomicAdd(&w.hist[b2.bin(v)], 1);
            });
            __syncwarp();
            int before2;
            cut_bin(w.hist, c - before, lane, &cut2, &before2);
            __syncwarp();
        }
    }
    auto keep = [&](float v) {
        const int bb = b1.bin(v);
        return bb < cut1 || (bb == cut1 && (b2.inv == 0.f || b2.bin(v) <= cut2));
    };
    int kept = 0;
    if constexpr (MODE == 2) {
        // in place: every lane reads its entry before any lane writes, and a
        // kept entry goes to a position at or before the one it came from
        for (int e0 = 0; e0 < total; e0 += 32) {
            const int e = e0 + lane;
            const uint64_t key = e < total ? w.keys[e] : 0ull;
            const bool take = e < total && keep(hit_val(static_cast<uint32_t>(key >> 32)));
            const unsigned bal = __ballot_sync(0xffffffffu, take);
            __syncwarp();
            const int pos = kept + __popc(bal & ((1u << lane) - 1u));
            if (take && pos < P) w.keys[pos] = static_cast<uint32_t>(key);
            kept += __popc(bal);
        }
    } else if constexpr (MODE == 1) {
        // compact the kept reference indices into w.keys in entry order (ballots)
#pragma unroll
        for (int i = 0; i < kRegHits; ++i) {
            const int e = i * 32 + lane;
            const bool take = e < total && keep(hit_val(hv[i]));
            const unsigned bal = __ballot_sync(0xffffffffu, take);
            const int pos = kept + __popc(bal & ((1u << lane) - 1u));
            if (take && pos < P) w.keys[pos] = static_cast<uint32_t>(w.stage[e]);
            kept += __popc(bal);
        }
    } else {
        if (lane == 0) w.hist[kBins] = 0;
        __syncwarp();
        visit_global([&](uint64_t key) {
            if (keep(hit_val(static_cast<uint32_t>(key >> 32)))) {
                const int pos = atomicAdd(&w.hist[kBins], 1);
                if (pos < P) w.keys[pos] = key_idx(key);
            }
        });
        __syncwarp();
        kept = w.hist[kBins];
    }
    __syncwarp();
    if (kept > P) return -3;
    exact_keys<METRIC, NV>(w.keys, kept, a.R, a.d, w.qrow, lane);
    return kept;
}

__device__ __forceinline__ void local_min(const uint64_t* keys, int pool, int lane, uint64_t* lmin,
                                          int* lpos) {
    uint64_t best = kEmptyKey;
    int at = -1;
    for (int e = lane; e < pool; e += 32) {
        const uint64_t v = keys[e];
        if (v < best) { best = v; at = e; }
    }
    *lmin = best;
    *lpos = at;
}

__device__ __forceinline__ uint64_t warp_min_key(uint64_t x) {
    const uint32_t hi = static_cast<uint32_t>(x >> 32);
    const uint32_t mhi = __reduce_min_sync(0xffffffffu, hi);
    const uint32_t lo = (hi == mhi) ? static_cast<uint32_t>(x) : 0xffffffffu;
    const uint32_t mlo = __reduce_min_sync(0xffffffffu, lo);
    return (static_cast<uint64_t>(mhi) << 32) | mlo;
}

__device__ __forceinline__ void cswap(uint64_t& a, uint64_t& b) {
    const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
    a = lo;
    b = hi;
}

__device__ __forceinline__ void queue_fallback(const FinalizeArgs& a, int64_t q, int reason) {
    const int pos = atomicAdd(a.fallback_count, 1);
    a.fallback_list[pos] = static_cast<int32_t>(q);
    if (a.fallback_total) atomicAdd(a.fallback_total, 1ull);
    if (a.fallback_reason) atomicAdd(&a.fallback_reason[reason], 1ull);
}

// Query q, start to end, by one warp (lane = its lane): scratch is the warp's
// shared memory (warp_scratch_bytes for these P, S, d and staging entries).
// Every step is warp-synchronous; nothing waits on the rest of the CTA.
template <int METRIC, int NV>
__device__ void finalize_query(const FinalizeArgs& a, int P, int stage_entries, int64_t q,
                               unsigned char* scratch, int lane) {
    const int S = a.use_hits ? 1 : a.cand.S;
    const int d = a.d, k = a.k;
    const int Lcap = prefix_cap(P, k);
    const int se = a.use_hits ? stage_entries : 0;   // staging entries (hit lists only)
    WarpScratch w = carve(scratch, P, Lcap, S, se);
    // entries that fit keys[P] and the staging area behind it (contiguous)
    const size_t union_bytes = prefix_bytes(Lcap) > static_cast<size_t>(se) * 8
                                   ? prefix_bytes(Lcap) : static_cast<size_t>(se) * 8;
    const int stage_all = static_cast<int>((align16(static_cast<size_t>(P) * 8) + union_bytes) / 8);
    // the query row: its loads are issued before the hit-list sizes are read
    const float* qg = a.Q + q * d;
    float4 qv = make_float4(0.f, 0.f, 0.f, 0.f);
    const bool qvec = NV > 0 && (reinterpret_cast<uintptr_t>(a.Q) & 15) == 0;
    if (qvec) {
        if (lane < (d >> 2)) qv = __ldg(reinterpret_cast<const float4*>(qg) + lane);
    } else {
        for (int t = lane; t < d; t += 32) w.qrow[t] = qg[t];
    }
    int total = 0, over = 0;
    if (a.use_hits) hit_totals(a, q, lane, &total, &over);
    if (qvec && lane < (d >> 2)) reinterpret_cast<float4*>(w.qrow)[lane] = qv;
    for (int s = lane; s < S; s += 32) w.smax[s] = 0;
    __syncwarp();

    // 1. candidates with exact float32 keys
    int pool;
    if (!a.use_hits) {
        pool = a.cand.S * a.cand.c;
        gather_cand<METRIC, NV>(a, q, w, lane);
    } else {
        if (over) pool = -2;
        else if (total < a.hits.c && total < a.m) pool = -1;
        else if (total <= kStage) pool = gather_hits_impl<METRIC, NV, 1>(a, q, P, w, lane, total);
        else if (total <= stage_all) pool = gather_hits_impl<METRIC, NV, 2>(a, q, P, w, lane, total);
        else pool = gather_hits_impl<METRIC, NV, 0>(a, q, P, w, lane, total);
        if (pool < 0) {
            if (lane == 0) queue_fallback(a, q, -pool - 1);
            return;
        }
    }
    __syncwarp();

    // 2. ascending prefix by repeated minimum: the first k, continued through
    //    the near-tie run holding position k-1
    const float relf = a.relf;
    int L = 0;
    uint64_t prev = 0;
    bool truncated = false;
    if (pool <= kRegPool) {
        // four keys per lane, sorted in registers; the owner of each warp
        // minimum shifts its next key up
        uint64_t kr[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = lane + 32 * i;
            kr[i] = (e < pool) ? w.keys[e] : kEmptyKey;
        }
        cswap(kr[0], kr[1]); cswap(kr[2], kr[3]); cswap(kr[0], kr[2]);
        cswap(kr[1], kr[3]); cswap(kr[1], kr[2]);
        __syncwarp();
        while (true) {
            const uint64_t win = warp_min_key(kr[0]);
            if (win == kEmptyKey) break;
            if (L >= k && !near_tie(key_dist(prev), key_dist(win), relf)) break;
            if (L == Lcap) { truncated = true; break; }   // run longer than the prefix holds
            if (kr[0] == win) {
                w.sorted[L] = win;
                kr[0] = kr[1]; kr[1] = kr[2]; kr[2] = kr[3]; kr[3] = kEmptyKey;
            }
            prev = win;
            ++L;
        }
    } else if (pool <= 32 * kSortedStripe) {
        // each lane sorts its stripe keys[lane + 32 j] in place (insertion
        // sort, at most kSortedStripe keys); then the owner of each warp
        // minimum just steps to the next key of its stripe
        const int nl = (pool - lane + 31) / 32;
        for (int j = 1; j < nl; ++j) {
            const uint64_t x = w.keys[lane + 32 * j];
            int i = j - 1;
            while (i >= 0 && w.keys[lane + 32 * i] > x) {
                w.keys[lane + 32 * (i + 1)] = w.keys[lane + 32 * i];
                --i;
            }
            w.keys[lane + 32 * (i + 1)] = x;
        }
        int pos = 0;
        uint64_t lmin = nl > 0 ? w.keys[lane] : kEmptyKey;
        while (true) {
            const uint64_t win = warp_min_key(lmin);
            if (win == kEmptyKey) break;
            if (L >= k && !near_tie(key_dist(prev), key_dist(win), relf)) break;
            if (L == Lcap) { truncated = true; break; }
            if (lmin == win) {
                w.sorted[L] = win;
                ++pos;
                lmin = pos < nl ? w.keys[lane + 32 * pos] : kEmptyKey;
            }
            prev = win;
            ++L;
        }
    } else {
        uint64_t lmin;
        int lpos;
        local_min(w.keys, pool, lane, &lmin, &lpos);
        while (true) {
            const uint64_t win = warp_min_key(lmin);
            if (win == kEmptyKey) break;
            if (L >= k && !near_tie(key_dist(prev), key_dist(win), relf)) break;
            if (L == Lcap) { truncated = true; break; }
            if (lmin == win) {                 // owner: take it, rescan
                w.sorted[L] = win;
                w.keys[lpos] = kEmptyKey;
                local_min(w.keys, pool, lane, &lmin, &lpos);
            }
            prev = win;
            ++L;
        }
    }
    __syncwarp();
    if (truncated) {
        if (lane == 0) queue_fallback(a, q, 3);
        return;
    }
    const int kk = min(k, L);

    // 3. re-check of near-tie runs inside the prefix
    bool any_tie = false;
    for (int p = 1 + lane; p < L; p += 32)
        any_tie |= near_tie(key_dist(w.sorted[p - 1]), key_dist(w.sorted[p]), relf);
    any_tie = __any_sync(0xffffffffu, any_tie);
    for (int p = lane; p < L; p += 32) w.runs[p] = -1;
    __syncwarp();
    // d64 of a re-checked entry: its float-float value (packed), or its float64
    // value when dbl (some run entry needed the float64 tier)
    bool dbl = false;
    if (any_tie) {
        if (lane == 0) {
            int p = 0, nr = 0;
            while (p < L) {
                int e = p;
                while (e + 1 < L && near_tie(key_dist(w.sorted[e]), key_dist(w.sorted[e + 1]), relf)) ++e;
                if (e > p)
                    for (int x = p; x <= e; ++x) { w.runs[x] = p; w.rend[x] = e; w.rlist[nr++] = x; }
                p = e + 1;
            }
            w.hist[kBins + 1] = nr;
        }
        __syncwarp();
        const int nr = w.hist[kBins + 1];
        // tier 1: float-float distances of every run entry
        refine_ff<METRIC, NV>(w, nr, a.R, d, lane);
        // tier 2: float64 (oracle arithmetic) where float-float cannot separate
        // an entry from a run neighbour
        uint64_t mark = 0;
        for (int p = lane, i = 0; p < L; p += 32, ++i) {
            const int s0 = w.runs[p];
            if (s0 < 0) continue;
            const uint64_t vp = w.d64[p];
            for (int x = s0; x <= w.rend[p]; ++x) {
                if (x == p) continue;
                const uint64_t vx = w.d64[x];
                const float diff = __fsub_rn(ff_hi(vx), ff_hi(vp)) + (ff_lo(vx) - ff_lo(vp));
                if (fabsf(diff) <= a.ffw * fmaxf(ff_hi(vx), ff_hi(vp)) + 1e-37f) { mark |= 1ull << i; break; }
            }
        }
        dbl = __any_sync(0xffffffffu, mark != 0);
        __syncwarp();
        if (dbl) {
            // rare: every run entry as a float64 value, exact float-float sums
            // or the oracle's own arithmetic for the marked ones
            for (int p = lane, i = 0; p < L; p += 32, ++i) {
                if (w.runs[p] < 0) continue;
                double v;
                if ((mark >> i) & 1ull) {
                    const uint32_t j = key_idx(w.sorted[p]);
                    v = dist_f64<METRIC>(w.qrow, a.R + static_cast<int64_t>(j) * d, d);
                } else {
                    v = static_cast<double>(ff_hi(w.d64[p])) + static_cast<double>(ff_lo(w.d64[p]));
                }
                w.d64[p] = dbits(v);
            }
        }
        __syncwarp();
        for (int p = lane; p < L; p += 32) {
            const int s0 = w.runs[p];
            if (s0 >= 0) {
                const uint64_t mine = w.d64[p];
                const uint32_t mj = key_idx(w.sorted[p]);
                int rank = 0;
                for (int x = s0; x <= w.rend[p]; ++x) {
                    const uint64_t o = w.d64[x];
                    const uint32_t oj = key_idx(w.sorted[x]);
                    const bool less = dbl ? (o < mine) : ff_less(o, mine);
                    rank += (less || (o == mine && oj < mj)) ? 1 : 0;
                }
                w.perm[s0 + rank] = p;
            }
        }
        __syncwarp();
        if (lane == 0 && nr > 0 && a.recheck_counter)
            atomicAdd(a.recheck_counter, static_cast<unsigned long long>(nr));
    }
    // refined distance of a re-checked entry
    auto refined = [&](uint64_t v) {
        return dbl ? static_cast<float>(bitsd(v)) : __fadd_rn(ff_hi(v), ff_lo(v));
    };
    auto source_of = [&](int s) { return (w.runs[s] >= 0) ? w.perm[s] : s; };

    // 4. completeness of a float32 candidate set: the references left out by a
    //    split have keys >= that split's largest kept key
    if (!a.use_hits && a.cand.exact && kk > 0) {
        const double rel = a.rel;
        const CandidateSet& cs = a.cand;
        bool have = false;
        double lower = 0.0;
        for (int s = 0; s < S; ++s) {
            const int64_t b = static_cast<int64_t>(s) * cs.chunk;
            const int64_t e = min(a.m, b + cs.chunk);
            if (e - b > cs.c) {
                const double v = static_cast<double>(key_dist(w.smax[s])) * (1.0 - rel);
                lower = have ? fmin(lower, v) : v;
                have = true;
            }
        }
        if (have) {
            const int sk = source_of(kk - 1);
            const double upper = (w.runs[kk - 1] >= 0)
                                     ? static_cast<double>(refined(w.d64[sk])) * (1.0 + 1e-6)
                                     : static_cast<double>(key_dist(w.sorted[sk])) * (1.0 + rel);
            if (!(lower > upper) || kk < k) {
                if (lane == 0) queue_fallback(a, q, 3);
                return;
            }
        }
    }

    // 5. outputs
    for (int s = lane; s < k; s += 32) {
        float dist = __int_as_float(0x7f800000);
        int32_t idx = -1;
        if (s < kk) {
            const int sp = source_of(s);
            idx = static_cast<int32_t>(key_idx(w.sorted[sp]));
            if (w.runs[s] >= 0) {
                const float v = refined(w.d64[sp]);
                dist = (METRIC == kL2) ? sqrtf(v) : v;
            } else {
                const float v = key_dist(w.sorted[sp]);
                dist = (METRIC == kL2) ? sqrtf(v) : v;
            }
        }
        a.dist_out[q * k + s] = dist;
        a.idx_out[q * k + s] = idx;
    }
}

template <int METRIC, int NV>
__global__ void __launch_bounds__(kFinThreads, 4)
finalize_kernel(FinalizeArgs a, int P, int warps_per_block, int stage_entries) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t q = static_cast<int64_t>(blockIdx.x) * warps_per_block + warp;
    if (a.fb_done && blockIdx.x == 0 && static_cast<int>(threadIdx.x) < a.fb_slots)
        a.fb_done[threadIdx.x] = 0;   // the fallback's chunk counters, for this search
    if (q >= a.n) return;   // warp-uniform: no block-level sync below
    const int S = a.use_hits ? 1 : a.cand.S;
    const size_t per_warp =
        warp_scratch_bytes(P, prefix_cap(P, a.k), S, a.d, a.use_hits ? stage_entries : 0);
    finalize_query<METRIC, NV>(a, P, stage_entries, q, smem_raw + per_warp * warp, lane);
}

// ---------------------------------------------------------------------------
// exact fallback (one CTA of 1024 threads per queued query): float32
// distances to every reference and the k-th smallest by radix selection on
// their bit patterns (four 8-bit passes, one shared-memory histogram per
// warp); every reference whose float32 distance could still place it in the
// answer (float32 <= kth * (1+e)/(1-e)) gets its float64 distance (the
// oracle's arithmetic); those are sorted by (float64 distance, index) and the
// first k written.  When more than kFbCand references qualify (masses of
// equal distances), the same selection runs over float64 keys of all m.
// ---------------------------------------------------------------------------
constexpr int kFbThreads = 1024;
constexpr int kFbWarps = kFbThreads / 32;
constexpr int kFbMaxK = 1024;
constexpr int kFbCand = 4096;
constexpr int64_t kFbChunk = 16384;   // references per CTA in the spread key pass
constexpr uint64_t kInfBits = 0x7ff0000000000000ull;

template <int NT>
struct FbShared {
    int hist[NT / 32][256];
    int digit, rank, cnt, less, taken;
    int wsum[NT / 32];
};

// Bin b of the summed per-warp histograms, and the digit whose cumulative
// count reaches `rank` (warp 0; the result goes to sh.digit / sh.rank).
template <int NT>
__device__ void pick_digit(FbShared<NT>& sh, int rank) {
    const int tid = threadIdx.x, lane = tid % 32;
    if (tid < 32) {
        int h[8], sum = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int v = 0;
            for (int w = 0; w < (NT / 32); ++w) v += sh.hist[w][8 * lane + i];
            h[i] = v;
            sum += v;
        }
        int incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        int cum = incl - sum;
        if (cum < rank && incl >= rank) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (cum + h[i] >= rank) {
                    sh.digit = 8 * lane + i;
                    sh.rank = rank - cum;
                    break;
                }
                cum += h[i];
            }
        }
    }
}

template <int NT>
__device__ void clear_hist(FbShared<NT>& sh) {
    for (int e = threadIdx.x; e < (NT / 32) * 256; e += NT) (&sh.hist[0][0])[e] = 0;
}

// k-th smallest (1-based rank k) of keys[0..m) in unsigned order.
template <int NT>
__device__ uint32_t radix_select32(const uint32_t* keys, int64_t m, int k, FbShared<NT>& sh) {
    const int tid = threadIdx.x, w = tid / 32;
    uint32_t prefix = 0, mask = 0;
    int rank = k;
    for (int shift = 24; shift >= 0; shift -= 8) {
        clear_hist<NT>(sh);
        __syncthreads();
        for (int64_t j = tid; j < m; j += NT) {
            const uint32_t u = keys[j];
            if ((u & mask) == prefix) atomicAdd(&sh.hist[w][(u >> shift) & 0xff], 1);
        }
        __syncthreads();
        pick_digit<NT>(sh, rank);
        __syncthreads();
        prefix |= static_cast<uint32_t>(sh.digit) << shift;
        mask |= 0xffu << shift;
        rank = sh.rank;
        __syncthreads();
    }
    return prefix;
}

// The same over non-negative doubles (bit patterns; eight passes); *ties =
// how many entries equal to the result belong to the first k.
template <int NT>
__device__ uint64_t radix_select64(const double* keys, int64_t m, int k, FbShared<NT>& sh, int* ties) {
    const int tid = threadIdx.x, w = tid / 32;
    uint64_t prefix = 0, mask = 0;
    int rank = k;
    for (int shift = 56; shift >= 0; shift -= 8) {
        clear_hist<NT>(sh);
        __syncthreads();
        for (int64_t j = tid; j < m; j += NT) {
            const uint64_t u = dbits(keys[j]);
            if ((u & mask) == prefix) atomicAdd(&sh.hist[w][(u >> shift) & 0xff], 1);
        }
        __syncthreads();
        pick_digit<NT>(sh, rank);
        __syncthreads();
        prefix |= static_cast<uint64_t>(sh.digit) << shift;
        mask |= 0xffull << shift;
        rank = sh.rank;
        __syncthreads();
    }
    *ties = rank;
    return prefix;
}

// Sort keys ck / indices ci [0..cnt) ascending by (key, index) in place
// (bitonic over the next power of two, padded with the largest pair).
template <int NT>
__device__ void sort_pairs(uint64_t* ck, uint32_t* ci, int cnt) {
    const int tid = threadIdx.x;
    int P2 = 1;
    while (P2 < cnt) P2 <<= 1;
    for (int i = cnt + tid; i < P2; i += NT) { ck[i] = ~0ull; ci[i] = 0xffffffffu; }
    __syncthreads();
    for (int size = 2; size <= P2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < P2; i += NT) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool gt = ck[i] > ck[j] || (ck[i] == ck[j] && ci[i] > ci[j]);
                    if (gt == ((i & size) == 0)) {
                        const uint64_t tk = ck[i]; ck[i] = ck[j]; ck[j] = tk;
                        const uint32_t tj = ci[i]; ci[i] = ci[j]; ci[j] = tj;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Float32 keys (distance bit patterns) of references [j_begin, j_end) of one
// query (row in shared memory) into keys32; four references per thread at a
// time, their loads issued together.
template <int METRIC, int NT>
__device__ void fb_keys(const FinalizeArgs& a, const float* qrow, uint32_t* keys32, int64_t j_begin,
                        int64_t j_end) {
    const int tid = threadIdx.x, d = a.d;
    const bool vec = ((d & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.R) & 15) == 0);
    for (int64_t j0 = j_begin + static_cast<int64_t>(tid) * 4; j0 < j_end; j0 += 4LL * NT) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        if (vec && j0 + 4 <= j_end) {
            const float4* q4 = reinterpret_cast<const float4*>(qrow);
            const float4* r4 = reinterpret_cast<const float4*>(a.R + j0 * d);
            const int d4 = d >> 2;
#pragma unroll 2
            for (int t = 0; t < d4; ++t) {
                const float4 y = q4[t];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float4 x = __ldg(r4 + u * d4 + t);
                    acc[u] = acc_f32<METRIC>(acc[u], y.x - x.x);
                    acc[u] = acc_f32<METRIC>(acc[u], y.y - x.y);
                    acc[u] = acc_f32<METRIC>(acc[u], y.z - x.z);
                    acc[u] = acc_f32<METRIC>(acc[u], y.w - x.w);
                }
            }
        } else {
            for (int u = 0; u < 4 && j0 + u < j_end; ++u)
                acc[u] = dist_f32<METRIC>(qrow, a.R + (j0 + u) * d, d);
        }
        for (int u = 0; u < 4 && j0 + u < j_end; ++u) keys32[j0 + u] = __float_as_uint(acc[u]);
    }
}

// Given the float32 keys of all m references of query q (keys32, aliasing the
// float64 scratch `keys`): the k-th by radix selection, float64 distances of
// every reference that could still be in the answer, the exact order and the
// k outputs.  One CTA.
template <int METRIC, int NT>
__device__ void fb_select(const FinalizeArgs& a, int64_t q, const float* qrow, double* keys,
                          uint32_t* keys32, FbShared<NT>& sh, uint64_t* ck, uint32_t* ci) {
    const int tid = threadIdx.x;
    const int64_t m = a.m;
    const int d = a.d, k = a.k;
    const double rel = f32_rel_bound(d);
    if (tid == 0) sh.cnt = 0;
    __syncthreads();
    const float kth32 = __uint_as_float(radix_select32<NT>(keys32, m, k, sh));
    const double bound = static_cast<double>(kth32) * (1.0 + rel) / (1.0 - rel) * (1.0 + 1e-12) + 1e-37;
    // the references that could still be in the answer, with float64 distances
    for (int64_t j = tid; j < m; j += NT) {
        if (static_cast<double>(__uint_as_float(keys32[j])) <= bound) {
            const int pos = atomicAdd(&sh.cnt, 1);
            if (pos < kFbCand) ci[pos] = static_cast<uint32_t>(j);
        }
    }
    __syncthreads();
    const int cnt = sh.cnt;
    if (cnt <= kFbCand) {
        for (int i = tid; i < cnt; i += NT)
            ck[i] = dbits(dist_f64<METRIC>(qrow, a.R + static_cast<int64_t>(ci[i]) * d, d));
        __syncthreads();
        sort_pairs<NT>(ck, ci, cnt);
    } else {
        // more candidates than shared memory holds: float64 keys of all m in
        // the scratch (they overwrite the float32 keys, so those are recomputed)
        for (int64_t j = tid; j < m; j += NT) {
            const float v32 = dist_f32<METRIC>(qrow, a.R + j * d, d);
            keys[j] = (static_cast<double>(v32) <= bound)
                          ? dist_f64<METRIC>(qrow, a.R + j * d, d)
                          : bitsd(kInfBits);
        }
        __syncthreads();
        int ties;
        const uint64_t T = radix_select64<NT>(keys, m, k, sh, &ties);
        const int n_less = k - ties;   // strictly below T; then `ties` entries equal to T
        if (tid == 0) { sh.less = 0; sh.taken = 0; }
        __syncthreads();
        for (int64_t j = tid; j < m; j += NT) {
            const uint64_t u = dbits(keys[j]);
            if (u < T) {
                const int slot = atomicAdd(&sh.less, 1);
                ck[slot] = u;
                ci[slot] = static_cast<uint32_t>(j);
            }
        }
        __syncthreads();
        // the `ties` entries equal to T with the smallest indices, in index order
        const int lane = tid % 32, wid = tid / 32;
        for (int64_t b0 = 0; b0 < m; b0 += NT) {
            const int64_t j = b0 + tid;
            const bool eq = (j < m) && dbits(keys[j]) == T;
            const unsigned bal = __ballot_sync(0xffffffffu, eq);
            if (lane == 0) sh.wsum[wid] = __popc(bal);
            __syncthreads();
            int before = sh.taken;
            for (int x = 0; x < wid; ++x) before += sh.wsum[x];
            before += __popc(bal & ((1u << lane) - 1u));
            if (eq && before < ties) {
                ck[n_less + before] = T;
                ci[n_less + before] = static_cast<uint32_t>(j);
            }
            __syncthreads();
            if (tid == 0) {
                int tot = 0;
                for (int x = 0; x < (NT / 32); ++x) tot += sh.wsum[x];
                sh.taken += tot;
            }
            __syncthreads();
            if (sh.taken >= ties) break;
        }
        sort_pairs<NT>(ck, ci, k);
    }
    for (int s = tid; s < k; s += NT) {
        const double v = bitsd(ck[s]);
        a.dist_out[q * k + s] =
            (METRIC == kL2) ? static_cast<float>(__dsqrt_rn(v)) : static_cast<float>(v);
        a.idx_out[q * k + s] = static_cast<int32_t>(ci[s]);
    }
}

// Shared-memory carve of the fallback kernels: candidate keys and indices,
// then the query row.
struct FbDyn {
    uint64_t* ck;
    uint32_t* ci;
    float* qrow;
};
__device__ __forceinline__ FbDyn fb_dyn_carve(unsigned char* base) {
    FbDyn f;
    f.ck = reinterpret_cast<uint64_t*>(base);                  // [kFbCand]
    f.ci = reinterpret_cast<uint32_t*>(f.ck + kFbCand);        // [kFbCand]
    f.qrow = reinterpret_cast<float*>(f.ci + kFbCand);         // [d + 4]
    return f;
}

// One launch for every queued query.  Rows y < spread of the grid: the first
// `spread` queued queries, spread over the GPU -- CTA (p, y) computes the
// float32 keys of chunk p (kFbChunk references) of queued query y into that
// query's scratch slot, and the CTA that completes a query's last chunk (a
// counter per slot, with fences around it) runs the selection; nothing waits
// on another CTA.  Rows y >= spread (column 0 only): the queued queries beyond
// the first `spread`, one CTA each, keys and selection, in scratch slot y.
// Queued query q, start to end, by one CTA of NT threads: its float32 keys
// of all m references into `keys` (a scratch row of m doubles), then the
// selection and the outputs.
template <int METRIC, int NT>
__device__ void fb_query(const FinalizeArgs& a, int64_t q, double* keys, FbShared<NT>& sh,
                         const FbDyn& f) {
    const int tid = threadIdx.x;
    uint32_t* keys32 = reinterpret_cast<uint32_t*>(keys);
    __syncthreads();
    for (int t = tid; t < a.d; t += NT) f.qrow[t] = a.Q[q * a.d + t];
    __syncthreads();
    fb_keys<METRIC, NT>(a, f.qrow, keys32, 0, a.m);
    __syncthreads();
    fb_select<METRIC, NT>(a, q, f.qrow, keys, keys32, sh, f.ck, f.ci);
    __syncthreads();
}

template <int METRIC>
__global__ void __launch_bounds__(kFbThreads)
fallback_kernel(FinalizeArgs a, double* __restrict__ scratch, int32_t* __restrict__ done,
                int32_t spread) {
    __shared__ FbShared<kFbThreads> sh;
    __shared__ int last;
    extern __shared__ __align__(16) unsigned char fb_dyn[];
    const FbDyn f = fb_dyn_carve(fb_dyn);
    const int tid = threadIdx.x;
    const int count = *a.fallback_count;
    const int y = blockIdx.y;
    const int64_t m = a.m;
    const int d = a.d;
    double* keys = scratch + static_cast<int64_t>(y) * m;
    uint32_t* keys32 = reinterpret_cast<uint32_t*>(keys);
    if (y < spread) {
        if (y >= count) return;   // CTA-uniform
        const int64_t q = a.fallback_list[y];
        for (int t = tid; t < d; t += kFbThreads) f.qrow[t] = a.Q[q * d + t];
        __syncthreads();
        const int64_t j0 = static_cast<int64_t>(blockIdx.x) * kFbChunk;
        fb_keys<METRIC, kFbThreads>(a, f.qrow, keys32, j0, min(m, j0 + kFbChunk));
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            last = (atomicAdd(&done[y], 1) == static_cast<int>(gridDim.x) - 1) ? 1 : 0;
        }
        __syncthreads();
        if (!last) return;
        __threadfence();
        fb_select<METRIC, kFbThreads>(a, q, f.qrow, keys, keys32, sh, f.ck, f.ci);
        if (tid == 0) done[y] = 0;
        return;
    }
    if (blockIdx.x != 0) return;
    const int tail = static_cast<int>(gridDim.y) - spread;
    for (int i = spread + (y - spread); i < count; i += tail) {
        const int64_t q = a.fallback_list[i];
        __syncthreads();
        for (int t = tid; t < d; t += kFbThreads) f.qrow[t] = a.Q[q * d + t];
        __syncthreads();
        fb_keys<METRIC, kFbThreads>(a, f.qrow, keys32, 0, m);
        __syncthreads();
        fb_select<METRIC, kFbThreads>(a, q, f.qrow, keys, keys32, sh, f.ck, f.ci);
    }
}

}  // namespace
}  // namespace knn
