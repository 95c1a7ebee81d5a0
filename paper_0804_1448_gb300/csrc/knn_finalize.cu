// knn_finalize.cu -- per-query completion of the search, and the exact fallback.
//
// finalize (one warp per query):
//   1. exact float32 distance of every candidate (differences, coordinate 0
//      first: the same arithmetic as the CUDA-core select kernel), which is
//      the "re-rank" of the tensor-core candidates;
//   2. sort by (distance, index) -- step 2 of the brute-force algorithm of
//      Sec. 2.1, restricted to the candidates;
//   3. near-tie re-check: consecutive candidates whose float32 distances are
//      closer than twice the float32 rounding bound can be out of exact order,
//      so every such run that reaches the first k positions is recomputed in
//      float64 (the oracle's arithmetic: widen, subtract, square or abs, add,
//      coordinate 0 first, no fused multiply-add) and re-ordered by
//      (float64 distance, index);
//   4. completeness check (float32 candidates only): the references that are
//      not candidates have float32 distances >= the largest key kept by their
//      split; if that bound, lowered by the rounding bound, does not exceed the
//      k-th exact distance, a non-candidate could still belong to the answer
//      and the query is queued for the fallback instead of being written;
//   5. the k outputs (Euclidean: square root of the squared distance).
//
// fallback (one CTA per queued query): float64 distances to all m references,
// exact radix selection of the k smallest (distance, index) pairs, sort, write.
#include "knn_internal.cuh"

namespace knn {
namespace {

constexpr int kMaxPool = 4096;

// Relative rounding bound of the float32 distance (squared Euclidean or
// Manhattan) accumulated over d coordinates with one rounding per difference
// and one per accumulation step: |d32 - d| <= (d + 2) u d, u = 2^-24.
// A safety factor of 2 covers the second-order terms.
__device__ __forceinline__ double f32_rel_bound(int d) {
    return 2.0 * (d + 2) * 5.9604644775390625e-8;
}

template <int METRIC>
__device__ __forceinline__ float dist_f32(const float* q, const float* __restrict__ r, int d) {
    float acc = 0.f;
    if ((d & 3) == 0) {   // rows are 16-byte aligned: vector loads, same order of operations
        const float4* r4 = reinterpret_cast<const float4*>(r);
        const float4* q4 = reinterpret_cast<const float4*>(q);
        for (int t = 0; t < d / 4; ++t) {
            const float4 x = __ldg(r4 + t);
            const float4 y = q4[t];
            const float e0 = y.x - x.x, e1 = y.y - x.y, e2 = y.z - x.z, e3 = y.w - x.w;
            if (METRIC == kL2) {
                acc = fmaf(e0, e0, acc); acc = fmaf(e1, e1, acc);
                acc = fmaf(e2, e2, acc); acc = fmaf(e3, e3, acc);
            } else {
                acc += fabsf(e0); acc += fabsf(e1); acc += fabsf(e2); acc += fabsf(e3);
            }
        }
        return acc;
    }
    for (int t = 0; t < d; ++t) {
        const float diff = q[t] - __ldg(r + t);
        if (METRIC == kL2) acc = fmaf(diff, diff, acc);
        else acc += fabsf(diff);
    }
    return acc;
}

// The oracle's float64 arithmetic, operation for operation.
template <int METRIC>
__device__ __forceinline__ double dist_f64(const float* q, const float* __restrict__ r, int d) {
    double acc = 0.0;
    for (int t = 0; t < d; ++t) {
        const double diff = __dsub_rn(static_cast<double>(q[t]), static_cast<double>(__ldg(r + t)));
        if (METRIC == kL2) acc = __dadd_rn(acc, __dmul_rn(diff, diff));
        else acc = __dadd_rn(acc, fabs(diff));
    }
    return acc;
}

__device__ __forceinline__ uint64_t dbits(double x) {
    return static_cast<uint64_t>(__double_as_longlong(x));
}
__device__ __forceinline__ double bitsd(uint64_t b) {
    return __longlong_as_double(static_cast<long long>(b));
}

// True when b (>= a) is within the float32 rounding of a, i.e. the exact
// order of the two can differ from their float32 order.
__device__ __forceinline__ bool near_tie(float a, float b, double rel) {
    return static_cast<double>(b) - static_cast<double>(a) <=
           2.0 * rel * static_cast<double>(b) + 1e-37;
}

struct WarpScratch {
    uint64_t* keys;  // [P] (float32 distance, index)
    uint64_t* d64;   // [P] float64 distance bits of re-checked entries
    int32_t* rs;     // [P] run start of re-checked entries, -1 otherwise
    int32_t* re;     // [P] run end (inclusive)
    int32_t* perm;   // [P] output position -> source position inside re-checked runs
    uint64_t* smax;  // [S] largest original key per split
    int32_t* hist;   // [kBins] histogram of hit-list keys; hist[kBins] = fill counter
    float* qrow;     // [d], 16-byte aligned
};

constexpr int kBins = 64;

__host__ __device__ inline size_t warp_scratch_bytes(int P, int S, int d) {
    const size_t b = static_cast<size_t>(P) * (8 + 8 + 4 + 4 + 4) + static_cast<size_t>((S + 1) & ~1) * 8 +
                     (kBins + 4) * 4 + (static_cast<size_t>(d) + 4) * 4;
    return (b + 15) & ~static_cast<size_t>(15);
}

// Hit-list front end: keep every listed reference whose low-precision key
// falls in the histogram bins up to the one holding rank c (so at least the
// best c), compute their exact float32 distances into w.keys, and return how
// many there are; -1 sends the query to the exact fallback.
template <int METRIC>
__device__ int gather_hits(const FinalizeArgs& a, int64_t q, int P, WarpScratch& w, int lane) {
    const HitLists& hl = a.hits;
    const int S = hl.S, cap = hl.cap;
    const int d = a.d;
    const uint64_t* base = hl.keys + q * static_cast<int64_t>(S) * cap;
    const int32_t* cnts = hl.counts + q * static_cast<int64_t>(S);
    int total = 0, over = 0;
    for (int s = lane; s < S; s += 32) {
        const int cs = cnts[s];
        over |= cs > cap;
        total += min(cs, cap);
    }
    for (int o = 16; o > 0; o >>= 1) {
        total += __shfl_xor_sync(0xffffffffu, total, o);
        over |= __shfl_xor_sync(0xffffffffu, over, o);
    }
    if (over) return -2;
    if (total < hl.c && total < a.m) return -1;
    // range of the order-mapped scores
    uint32_t omin = 0xffffffffu, omax = 0;
    for (int s = 0; s < S; ++s) {
        const int cs = min(cnts[s], cap);
        for (int e = lane; e < cs; e += 32) {
            const uint32_t o = static_cast<uint32_t>(base[static_cast<int64_t>(s) * cap + e] >> 32);
            omin = min(omin, o);
            omax = max(omax, o);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        omin = min(omin, __shfl_xor_sync(0xffffffffu, omin, o));
        omax = max(omax, __shfl_xor_sync(0xffffffffu, omax, o));
    }
    const uint64_t span = static_cast<uint64_t>(omax) - omin + 1;
    int cut = kBins - 1;            // keep bins 0..cut
    if (total > hl.c) {
        for (int b = lane; b < kBins + 4; b += 32) w.hist[b] = 0;
        __syncwarp();
        for (int s = 0; s < S; ++s) {
            const int cs = min(cnts[s], cap);
            for (int e = lane; e < cs; e += 32) {
                const uint32_t o = static_cast<uint32_t>(base[static_cast<int64_t>(s) * cap + e] >> 32);
                atomicAdd(&w.hist[static_cast<int>((static_cast<uint64_t>(o - omin) * kBins) / span)], 1);
            }
        }
        __syncwarp();
        // smallest bin whose cumulative count reaches c (two bins per lane)
        const int h0 = w.hist[2 * lane], h1 = w.hist[2 * lane + 1];
        int incl = h0 + h1;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int excl = incl - h0 - h1;
        int mine = kBins;
        if (excl + h0 >= hl.c) mine = 2 * lane;
        else if (incl >= hl.c) mine = 2 * lane + 1;
        for (int o = 16; o > 0; o >>= 1) mine = min(mine, __shfl_xor_sync(0xffffffffu, mine, o));
        cut = mine;
    }
    // keep, re-rank in float32
    if (lane == 0) w.hist[kBins] = 0;
    __syncwarp();
    int kept = 0;
    for (int s = 0; s < S; ++s) {
        const int cs = min(cnts[s], cap);
        for (int e0 = 0; e0 < cs; e0 += 32) {
            const int e = e0 + lane;
            bool take = false;
            uint32_t j = 0;
            if (e < cs) {
                const uint64_t key = base[static_cast<int64_t>(s) * cap + e];
                const uint32_t o = static_cast<uint32_t>(key >> 32);
                take = static_cast<int>((static_cast<uint64_t>(o - omin) * kBins) / span) <= cut;
                j = key_idx(key);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, take);
            const int pos = kept + __popc(bal & ((1u << lane) - 1u));
            if (take && pos < P)
                w.keys[pos] = make_key(dist_f32<METRIC>(w.qrow, a.R + static_cast<int64_t>(j) * d, d), j);
            kept += __popc(bal);
        }
    }
    __syncwarp();
    return kept <= P ? kept : -3;
}

template <int METRIC>
__global__ void finalize_kernel(FinalizeArgs a, int P, int warps_per_block) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t q = static_cast<int64_t>(blockIdx.x) * warps_per_block + warp;
    if (q >= a.n) return;   // warp-uniform: no block-level sync below

    const CandidateSet& cs = a.cand;
    const int S = a.use_hits ? 1 : cs.S, c = cs.c, Sc = a.use_hits ? 0 : S * c;
    const int d = a.d;
    const size_t per_warp = warp_scratch_bytes(P, S, d);
    unsigned char* base = smem_raw + per_warp * warp;
    WarpScratch w;
    w.keys = reinterpret_cast<uint64_t*>(base);
    w.d64 = w.keys + P;
    w.smax = w.d64 + P;
    w.rs = reinterpret_cast<int32_t*>(w.smax + ((S + 1) & ~1));
    w.re = w.rs + P;
    w.perm = w.re + P;
    w.hist = w.perm + P;
    w.qrow = reinterpret_cast<float*>(w.hist + kBins + 4);

    for (int t = lane; t < d; t += 32) w.qrow[t] = a.Q[q * d + t];
    for (int s = lane; s < S; s += 32) w.smax[s] = 0;
    for (int e = lane; e < P; e += 32) { w.keys[e] = kEmptyKey; w.rs[e] = -1; }
    __syncwarp();

    // 1. exact float32 distances of the candidates
    int cnt = 0;
    if (!a.use_hits) {
        const uint64_t* src = cs.keys + q * static_cast<int64_t>(Sc);
        for (int e0 = 0; e0 < Sc; e0 += 32) {
            const int e = e0 + lane;
            uint64_t nk = kEmptyKey;
            if (e < Sc) {
                const uint64_t key = src[e];
                if (key != kEmptyKey) {
                    const uint32_t j = key_idx(key);
                    nk = make_key(dist_f32<METRIC>(w.qrow, a.R + static_cast<int64_t>(j) * d, d), j);
                    atomicMax(reinterpret_cast<unsigned long long*>(&w.smax[e / c]),
                              static_cast<unsigned long long>(key));
                }
                w.keys[e] = nk;
            }
            cnt += __popc(__ballot_sync(0xffffffffu, nk != kEmptyKey));
        }
    } else {
        cnt = gather_hits<METRIC>(a, q, P, w, lane);
        if (cnt < 0) {   // -1 short list, -2 overflow, -3 the cut kept too many
            if (lane == 0) {
                const int pos = atomicAdd(a.fallback_count, 1);
                a.fallback_list[pos] = static_cast<int32_t>(q);
                if (a.fallback_total) atomicAdd(a.fallback_total, 1ull);
                if (a.fallback_reason) atomicAdd(&a.fallback_reason[-cnt - 1], 1ull);
            }
            return;
        }
    }
    __syncwarp();

    // 2. bitonic sort by (distance, index)
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < P; i += 32) {
                const int j = i ^ stride;
                if (j > i) {
                    const uint64_t x = w.keys[i], y = w.keys[j];
                    const bool up = (i & size) == 0;
                    if ((x > y) == up) { w.keys[i] = y; w.keys[j] = x; }
                }
            }
            __syncwarp();
        }
    }

    const int k = a.k;
    const int kk = min(k, cnt);
    const double rel = f32_rel_bound(d);

    // 3a. find the near-tie runs that reach the first kk positions (lane 0)
    int scan_end = 0;
    if (lane == 0 && kk > 0) {
        int p = 0;
        while (p < kk) {
            int e = p;
            while (e + 1 < cnt && near_tie(key_dist(w.keys[e]), key_dist(w.keys[e + 1]), rel)) ++e;
            if (e > p) {
                for (int x = p; x <= e; ++x) { w.rs[x] = p; w.re[x] = e; }
            }
            p = e + 1;
        }
        scan_end = p;   // one past the last position of the run holding kk-1
    }
    scan_end = __shfl_sync(0xffffffffu, scan_end, 0);
    __syncwarp();

    // 3b. float64 distances of re-checked entries, then their rank in the run
    int nre = 0;
    for (int p = lane; p < scan_end; p += 32) {
        if (w.rs[p] >= 0) {
            const uint32_t j = key_idx(w.keys[p]);
            w.d64[p] = dbits(dist_f64<METRIC>(w.qrow, a.R + static_cast<int64_t>(j) * d, d));
            ++nre;
        }
    }
    __syncwarp();
    for (int p = lane; p < scan_end; p += 32) {
        const int s0 = w.rs[p];
        if (s0 >= 0) {
            const uint64_t mine = w.d64[p];
            const uint32_t mj = key_idx(w.keys[p]);
            int rank = 0;
            for (int x = s0; x <= w.re[p]; ++x) {
                const uint64_t o = w.d64[x];
                const uint32_t oj = key_idx(w.keys[x]);
                rank += (o < mine || (o == mine && oj < mj)) ? 1 : 0;
            }
            w.perm[s0 + rank] = p;
        }
    }
    __syncwarp();
    for (int o = 16; o > 0; o >>= 1) nre += __shfl_xor_sync(0xffffffffu, nre, o);
    if (lane == 0 && nre > 0 && a.recheck_counter)
        atomicAdd(a.recheck_counter, static_cast<unsigned long long>(nre));

    auto source_of = [&](int s) { return (w.rs[s] >= 0) ? w.perm[s] : s; };

    // 4. completeness of a float32 candidate set
    if (!a.use_hits && cs.exact && kk > 0) {
        bool have = false;
        double lower = 0.0;
        for (int s = 0; s < S; ++s) {
            const int64_t b = static_cast<int64_t>(s) * cs.chunk;
            const int64_t e = min(a.m, b + cs.chunk);
            if (e - b > c) {   // this split left references out
                const double v = static_cast<double>(key_dist(w.smax[s])) * (1.0 - rel);
                lower = have ? fmin(lower, v) : v;
                have = true;
            }
        }
        if (have) {
            const int sk = source_of(kk - 1);
            const double upper = (w.rs[kk - 1] >= 0)
                                     ? bitsd(w.d64[sk])
                                     : static_cast<double>(key_dist(w.keys[sk])) * (1.0 + rel);
            if (!(lower > upper) || kk < k) {
                if (lane == 0) {
                    const int pos = atomicAdd(a.fallback_count, 1);
                    a.fallback_list[pos] = static_cast<int32_t>(q);
                    if (a.fallback_total) atomicAdd(a.fallback_total, 1ull);
                    if (a.fallback_reason) atomicAdd(&a.fallback_reason[3], 1ull);
                }
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
            idx = static_cast<int32_t>(key_idx(w.keys[sp]));
            if (w.rs[s] >= 0) {
                const double v = bitsd(w.d64[sp]);
                dist = (METRIC == kL2) ? static_cast<float>(__dsqrt_rn(v)) : static_cast<float>(v);
            } else {
                const float v = key_dist(w.keys[sp]);
                dist = (METRIC == kL2) ? sqrtf(v) : v;
            }
        }
        a.dist_out[q * k + s] = dist;
        a.idx_out[q * k + s] = idx;
    }
}

// ---------------------------------------------------------------------------
// exact float64 fallback
// ---------------------------------------------------------------------------
constexpr int kFbThreads = 256;
constexpr int kFbMaxK = 1024;

template <int METRIC>
__global__ void __launch_bounds__(kFbThreads)
fallback_kernel(FinalizeArgs a, double* __restrict__ scratch) {
    __shared__ int hist[256];
    __shared__ uint64_t ck[kFbMaxK];
    __shared__ uint32_t ci[kFbMaxK];
    __shared__ int s_digit, s_rank, s_less, s_taken, s_wsum[kFbThreads / 32];
    extern __shared__ float qrow[];

    const int tid = threadIdx.x;
    const int count = *a.fallback_count;
    const int64_t m = a.m;
    const int d = a.d, k = a.k;
    double* keys = scratch + static_cast<int64_t>(blockIdx.x) * m;

    for (int f = blockIdx.x; f < count; f += gridDim.x) {
        const int64_t q = a.fallback_list[f];
        __syncthreads();
        for (int t = tid; t < d; t += kFbThreads) qrow[t] = a.Q[q * d + t];
        __syncthreads();
        for (int64_t j = tid; j < m; j += kFbThreads)
            keys[j] = dist_f64<METRIC>(qrow, a.R + j * d, d);
        __syncthreads();

        // radix selection of the k-th smallest key (non-negative doubles:
        // the bit pattern orders like the value)
        uint64_t prefix = 0, mask = 0;
        int rank = k;
        for (int shift = 56; shift >= 0; shift -= 8) {
            for (int b = tid; b < 256; b += kFbThreads) hist[b] = 0;
            __syncthreads();
            for (int64_t j = tid; j < m; j += kFbThreads) {
                const uint64_t u = dbits(keys[j]);
                if ((u & mask) == prefix) atomicAdd(&hist[(u >> shift) & 0xff], 1);
            }
            __syncthreads();
            if (tid == 0) {
                int cum = 0, b = 0;
                for (; b < 256; ++b) {
                    if (cum + hist[b] >= rank) break;
                    cum += hist[b];
                }
                s_digit = b;
                s_rank = rank - cum;
            }
            __syncthreads();
            prefix |= static_cast<uint64_t>(s_digit) << shift;
            mask |= 0xffull << shift;
            rank = s_rank;
            __syncthreads();
        }
        const uint64_t T = prefix;   // bits of the k-th smallest distance
        const int n_less = k - rank; // entries strictly below T; then `rank` ties at T
        if (tid == 0) { s_less = 0; s_taken = 0; }
        __syncthreads();
        for (int64_t j = tid; j < m; j += kFbThreads) {
            const uint64_t u = dbits(keys[j]);
            if (u < T) {
                const int slot = atomicAdd(&s_less, 1);
                ck[slot] = u;
                ci[slot] = static_cast<uint32_t>(j);
            }
        }
        __syncthreads();
        // the `rank` ties at T with the smallest indices, in index order
        for (int64_t base = 0; base < m; base += kFbThreads) {
            const int64_t j = base + tid;
            const bool eq = (j < m) && dbits(keys[j]) == T;
            const unsigned bal = __ballot_sync(0xffffffffu, eq);
            const int lane = tid % 32, wid = tid / 32;
            if (lane == 0) s_wsum[wid] = __popc(bal);
            __syncthreads();
            int before = s_taken;
            for (int x = 0; x < wid; ++x) before += s_wsum[x];
            before += __popc(bal & ((1u << lane) - 1u));
            if (eq && before < rank) {
                ck[n_less + before] = T;
                ci[n_less + before] = static_cast<uint32_t>(j);
            }
            __syncthreads();
            if (tid == 0) {
                int tot = 0;
                for (int x = 0; x < kFbThreads / 32; ++x) tot += s_wsum[x];
                s_taken += tot;
            }
            __syncthreads();
            if (s_taken >= rank) break;
        }
        // sort the k selected pairs by (distance, index)
        int P2 = 1;
        while (P2 < k) P2 <<= 1;
        for (int i = k + tid; i < P2; i += kFbThreads) { ck[i] = ~0ull; ci[i] = 0xffffffffu; }
        __syncthreads();
        for (int size = 2; size <= P2; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = tid; i < P2; i += kFbThreads) {
                    const int j = i ^ stride;
                    if (j > i) {
                        const bool gt = ck[i] > ck[j] || (ck[i] == ck[j] && ci[i] > ci[j]);
                        const bool up = (i & size) == 0;
                        if (gt == up) {
                            const uint64_t tk = ck[i]; ck[i] = ck[j]; ck[j] = tk;
                            const uint32_t tj = ci[i]; ci[i] = ci[j]; ci[j] = tj;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int s = tid; s < k; s += kFbThreads) {
            const double v = bitsd(ck[s]);
            a.dist_out[q * k + s] =
                (METRIC == kL2) ? static_cast<float>(__dsqrt_rn(v)) : static_cast<float>(v);
            a.idx_out[q * k + s] = static_cast<int32_t>(ci[s]);
        }
    }
}

}  // namespace

int finalize_max_pool() { return kMaxPool; }

cudaError_t launch_finalize(const FinalizeArgs& a, cudaStream_t st, int* launches) {
    const int want = a.use_hits ? 2 * a.hits.c + 32 : a.cand.S * a.cand.c;
    int P = 32;
    while (P < want) P <<= 1;
    if (P > kMaxPool) return cudaErrorInvalidValue;
    const size_t per_warp = warp_scratch_bytes(P, a.use_hits ? 1 : a.cand.S, a.d);
    int wpb = static_cast<int>((48 * 1024) / per_warp);
    wpb = wpb < 1 ? 1 : (wpb > 8 ? 8 : wpb);
    const size_t smem = per_warp * wpb;
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    const unsigned grid = static_cast<unsigned>((a.n + wpb - 1) / wpb);
    if (launches) ++*launches;
    if (a.metric == kL2) {
        cudaError_t err = cudaFuncSetAttribute(finalize_kernel<kL2>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(smem));
        if (err != cudaSuccess) return err;
        finalize_kernel<kL2><<<grid, wpb * 32, smem, st>>>(a, P, wpb);
    } else {
        cudaError_t err = cudaFuncSetAttribute(finalize_kernel<kL1>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(smem));
        if (err != cudaSuccess) return err;
        finalize_kernel<kL1><<<grid, wpb * 32, smem, st>>>(a, P, wpb);
    }
    return cudaGetLastError();
}

cudaError_t launch_fallback(const FinalizeArgs& a, double* scratch, int32_t grid,
                            cudaStream_t st, int* launches) {
    if (a.k > kFbMaxK) return cudaErrorInvalidValue;
    const size_t smem = static_cast<size_t>(a.d) * sizeof(float);
    if (launches) ++*launches;
    if (a.metric == kL2)
        fallback_kernel<kL2><<<grid, kFbThreads, smem, st>>>(a, scratch);
    else
        fallback_kernel<kL1><<<grid, kFbThreads, smem, st>>>(a, scratch);
    return cudaGetLastError();
}

}  // namespace knn
