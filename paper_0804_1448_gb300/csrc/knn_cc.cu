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

// Shared memory: the two coordinate-stage buffers (queries and references)
// and the finished distance tile use the same space, one after the other;
// the heaps follow.
template <int ROWS>
constexpr size_t cc_stage_bytes() {
    return sizeof(float) * 2 * kDK * ((ROWS + 4) + (kTM + 4));
}
template <int ROWS>
constexpr size_t cc_union_bytes() {
    return cc_stage_bytes<ROWS>() > sizeof(float) * ROWS * (kTM + 1)
               ? cc_stage_bytes<ROWS>()
               : sizeof(float) * ROWS * (kTM + 1);
}
template <int ROWS>
constexpr size_t cc_smem_bytes(int c) {
    return cc_union_bytes<ROWS>() + sizeof(uint64_t) * static_cast<size_t>(c) * ROWS;
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

// Two float32 lanes: (a, a) - (b0, b1), the difference of one query
// coordinate and the same coordinate of two references, rounded per lane.
__device__ __forceinline__ uint64_t sub_pair(float a, float b0, float b1) {
    uint64_t r;
    asm("{\n .reg .b64 x, y;\n mov.b64 x, {%1, %1};\n mov.b64 y, {%2, %3};\n"
        " sub.rn.f32x2 %0, x, y;\n}"
        : "=l"(r) : "f"(a), "f"(b0), "f"(b1));
    return r;
}
// acc + diff * diff per lane, one rounding (the fmaf of the scalar form).
__device__ __forceinline__ uint64_t sqacc_pair(uint64_t diff, uint64_t acc) {
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(r) : "l"(diff), "l"(acc));
    return r;
}
__device__ __forceinline__ float pair_lo(uint64_t v) { return __uint_as_float(static_cast<uint32_t>(v)); }
__device__ __forceinline__ float pair_hi(uint64_t v) { return __uint_as_float(static_cast<uint32_t>(v >> 32)); }

// The (tile, coordinate stage) steps of a CTA run as one sequence h: step h
// reads the coordinates [16k, 16k + 16) (k = h % stages) of the queries and
// of reference tile h / stages.  Each thread loads its share of step h + 1
// from global memory into registers before it works on step h, so the loads
// are in flight during the arithmetic; two shared-memory buffers alternate,
// and one barrier per step separates the writes of a buffer from the reads of
// the step before.  A finished tile's distances take the buffers' place until
// the selector threads have consumed them (two more barriers per tile).
// Euclidean sums run as two-lane float32 instructions (sub, fma): per lane
// the same operations, in the same order, as the scalar form.
template <int METRIC, int ROWS>
__global__ void __launch_bounds__(kThreads, 3)
cc_select_kernel(const float* __restrict__ Q, int64_t n, const float* __restrict__ R,
                 int64_t m, int32_t d, CandidateSet cand) {
    using S = CCShape<ROWS>;
    static_assert(S::TY * S::TX == kThreads, "thread shape");
    static_assert(S::TY * S::RR == ROWS && S::TX * S::CN == kTM, "tile shape");
    static_assert(S::CN % 2 == 0 && S::G % 2 == 0, "column pairs");
    constexpr int QST = ROWS + 4;      // padded strides (bank spread)
    constexpr int RST = kTM + 4;
    constexpr int DST = kTM + 1;
    constexpr int QPT = ROWS * kDK / kThreads;   // query values per thread and step
    constexpr int RPT = kTM * kDK / kThreads;    // reference values per thread and step
    constexpr int CP = S::CN / 2;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Qs = reinterpret_cast<float*>(smem_raw);            // [2][kDK][QST]
    float* Rs = Qs + 2 * kDK * QST;                            // [2][kDK][RST]
    float* Dt = reinterpret_cast<float*>(smem_raw);            // [ROWS][DST], over the stages
    uint64_t* heap = reinterpret_cast<uint64_t*>(smem_raw + cc_union_bytes<ROWS>());  // [c][ROWS]

    const int tid = threadIdx.x;
    const int ty = tid / S::TX, tx = tid % S::TX;
    const int c = cand.c;
    const int64_t qbase = static_cast<int64_t>(blockIdx.x) * ROWS;
    const int split = blockIdx.y;
    const int64_t r_begin = static_cast<int64_t>(split) * cand.chunk;
    const int64_t r_end = min(m, r_begin + cand.chunk);
    const int stages = (d + kDK - 1) / kDK;
    const int tiles = r_end > r_begin ? static_cast<int>((r_end - r_begin + kTM - 1) / kTM) : 0;
    const int steps = tiles * stages;

    for (int e = tid; e < c * ROWS; e += kThreads) heap[e] = kEmptyKey;
    uint64_t top = kEmptyKey;  // cached heap[0] of this thread's row (selector threads)
    float top_d = __int_as_float(0x7f800000);   // its distance (+inf while the heap has room)

    float pq[QPT], pr[RPT];
    auto fetch = [&](int h) {
        const int64_t tbase = r_begin + static_cast<int64_t>(h / stages) * kTM;
        const int dbase = (h % stages) * kDK;
#pragma unroll
        for (int u = 0; u < QPT; ++u) {
            const int e = tid + u * kThreads, r = e / kDK, t = e % kDK;
            const int64_t gq = qbase + r;
            const int gt = dbase + t;
            pq[u] = (gq < n && gt < d) ? Q[gq * d + gt] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int e = tid + u * kThreads, r = e / kDK, t = e % kDK;
            const int64_t gr = tbase + r;
            const int gt = dbase + t;
            pr[u] = (gr < r_end && gt < d) ? R[gr * d + gt] : 0.f;
        }
    };
    if (steps > 0) fetch(0);

    float acc[S::RR][S::CN];
    uint64_t acc2[S::RR][CP];
#pragma unroll
    for (int i = 0; i < S::RR; ++i) {
#pragma unroll
        for (int j = 0; j < S::CN; ++j) acc[i][j] = 0.f;
#pragma unroll
        for (int j = 0; j < CP; ++j) acc2[i][j] = 0ull;
    }

    for (int h = 0; h < steps; ++h) {
        float* qs = Qs + (h & 1) * kDK * QST;
        float* rs = Rs + (h & 1) * kDK * RST;
#pragma unroll
        for (int u = 0; u < QPT; ++u) {
            const int e = tid + u * kThreads;
            qs[(e % kDK) * QST + e / kDK] = pq[u];
        }
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int e = tid + u * kThreads;
            rs[(e % kDK) * RST + e / kDK] = pr[u];
        }
        __syncthreads();
        if (h + 1 < steps) fetch(h + 1);
#pragma unroll 4
        for (int t = 0; t < kDK; ++t) {
            float qv[S::RR], rv[S::CN];
            const float4 q4 = *reinterpret_cast<const float4*>(&qs[t * QST + ty * S::RR]);
            qv[0] = q4.x; qv[1] = q4.y; qv[2] = q4.z; qv[3] = q4.w;
#pragma unroll
            for (int g = 0; g < S::CN / S::G; ++g) {
                const float* src = &rs[t * RST + g * S::TX * S::G + tx * S::G];
                if constexpr (S::G == 4) {
                    const float4 r4 = *reinterpret_cast<const float4*>(src);
                    rv[g * 4 + 0] = r4.x; rv[g * 4 + 1] = r4.y;
                    rv[g * 4 + 2] = r4.z; rv[g * 4 + 3] = r4.w;
                } else {
                    const float2 r2 = *reinterpret_cast<const float2*>(src);
                    rv[g * 2 + 0] = r2.x; rv[g * 2 + 1] = r2.y;
                }
            }
            if constexpr (METRIC == kL2) {
#pragma unroll
                for (int i = 0; i < S::RR; ++i)
#pragma unroll
                    for (int j = 0; j < CP; ++j)
                        acc2[i][j] = sqacc_pair(sub_pair(qv[i], rv[2 * j], rv[2 * j + 1]), acc2[i][j]);
            } else {
#pragma unroll
                for (int i = 0; i < S::RR; ++i)
#pragma unroll
                    for (int j = 0; j < S::CN; ++j) {
                        const float diff = qv[i] - rv[j];
                        if (METRIC == kL1) acc[i][j] += fabsf(diff);
                        else acc[i][j] = fmaxf(acc[i][j], fabsf(diff));
                    }
            }
        }
        if (h % stages != stages - 1) continue;

        // a reference tile is complete: its distances -> shared memory, over
        // the stage buffers once every thread is done reading them
        const int64_t tbase = r_begin + static_cast<int64_t>(h / stages) * kTM;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < S::RR; ++i)
#pragma unroll
            for (int j = 0; j < S::CN; ++j) {
                const int col = (j / S::G) * (S::TX * S::G) + tx * S::G + (j % S::G);
                float v;
                if constexpr (METRIC == kL2) v = (j & 1) ? pair_hi(acc2[i][j / 2]) : pair_lo(acc2[i][j / 2]);
                else v = acc[i][j];
                Dt[(ty * S::RR + i) * DST + col] = v;
                acc[i][j] = 0.f;
            }
#pragma unroll
        for (int i = 0; i < S::RR; ++i)
#pragma unroll
            for (int j = 0; j < CP; ++j) acc2[i][j] = 0ull;
        __syncthreads();
        // one thread per query row streams the tile through the row's heap;
        // a distance above the heap's largest cannot enter it (four columns
        // read ahead, so their loads overlap)
        if (tid < ROWS && qbase + tid < n) {
            uint64_t* hp = heap + tid;
            const int cols = static_cast<int>(min(static_cast<int64_t>(kTM), r_end - tbase));
            const float* drow = Dt + tid * DST;
            for (int c0 = 0; c0 < cols; c0 += 4) {
                float v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = (c0 + u < cols) ? drow[c0 + u] : top_d;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (c0 + u < cols && v[u] <= top_d) {
                        const uint64_t key = make_key(v[u], static_cast<uint32_t>(tbase + c0 + u));
                        if (key < top) {
                            heap_replace_top<ROWS>(hp, c, key);
                            top = hp[0];
                            top_d = top == kEmptyKey ? __int_as_float(0x7f800000) : key_dist(top);
                        }
                    }
                }
            }
        }
        __syncthreads();   // the tile is consumed: the next step's stores may overwrite it
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
constexpr size_t kSmemPerSm = 233472;   // shared memory of one SM
constexpr size_t kSmemPerCta = 1024;    // reserved by the hardware per resident CTA
constexpr int kMaxResident = 3;         // CTAs per SM the register bound allows

}  // namespace

int cc_plan_splits(int64_t n, int64_t m, int32_t c, int num_sms, int max_pool,
                   int64_t* chunk_out) {
    const bool wide = cc_smem_bytes<64>(c) <= kSmemCap;
    const int64_t rows = wide ? 64 : 16;
    const size_t smem = wide ? cc_smem_bytes<64>(c) : cc_smem_bytes<16>(c);
    int64_t per_sm = static_cast<int64_t>(kSmemPerSm / (smem + kSmemPerCta));
    if (per_sm > kMaxResident) per_sm = kMaxResident;
    if (per_sm < 1) per_sm = 1;
    const int64_t sms = num_sms > 0 ? num_sms : 1;
    const int64_t slots = per_sm * sms;
    const int64_t tiles = n > 0 ? (n + rows - 1) / rows : 1;
    int64_t s_cap = m / (8LL * c);                       // every split much longer than c
    if (s_cap > max_pool / c) s_cap = max_pool / c;      // all candidates in one finalize pool
    if (s_cap < 1) s_cap = 1;
    // Time with S splits, in units of one reference streamed by one CTA with
    // the SM to itself (the CTAs resident on an SM share its throughput): the
    // full waves take per_sm CTAs per SM, the last one the most CTAs any SM
    // gets, each CTA streaming its chunk plus two tiles' worth for its start
    // and end.  The smallest S within 2% of the best estimate wins.
    auto chunk_of = [&](int64_t S) { return ((m + S - 1) / S + kTM - 1) / kTM * kTM; };
    auto cost = [&](int64_t S) {
        const int64_t chunk = chunk_of(S), Sr = (m + chunk - 1) / chunk;
        const int64_t ctas = tiles * Sr;
        const int64_t rounds = (ctas / slots) * per_sm + (ctas % slots + sms - 1) / sms;
        return static_cast<double>(rounds) * static_cast<double>(chunk + 2 * kTM);
    };
    // The estimate takes a lone CTA on an SM to run as fast as the SM's full
    // share, which holds for long chunks only; when the query tiles give
    // fewer than two CTAs per SM, at least enough splits for two are taken.
    int64_t s_min = 1;
    if (tiles < 2 * sms) s_min = (2 * sms + tiles - 1) / tiles;
    if (s_min > s_cap) s_min = s_cap;
    double best = cost(s_min);
    for (int64_t S = s_min + 1; S <= s_cap; ++S) best = best < cost(S) ? best : cost(S);
    int64_t S = s_min;
    while (S < s_cap && cost(S) > 1.02 * best) ++S;
    const int64_t chunk = chunk_of(S);
    *chunk_out = chunk;
    return static_cast<int>((m + chunk - 1) / chunk);
}

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
