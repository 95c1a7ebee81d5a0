// knn_cc.cu -- float32 CUDA-core fused distance + per-query top-c selection.
//
// Step 1 of the brute-force algorithm of Sec. 2.1 (all distances between q_i
// and the r_j) fused with steps 2-3 (sort, keep the smallest): a CTA owns
// ROWS queries and streams the references of its split through shared memory
// in tiles of TM; each thread accumulates an RR x CN register micro-tile of
// distances over the d coordinates; the finished tile goes to shared memory.
// Selection is warp-level: every thread of the CTA tests its share of one
// query row's tile against that row's current threshold (the largest key of
// the row's bounded max-heap of c candidates), the pass bits of a row are
// gathered by warp shuffles into the row's leader lane, and the leader inserts
// only the passing distances.  After the first tiles almost nothing passes,
// so the serial part of the selection shrinks to the rare insertions.  Only
// the c survivors per (query, split) are written out.
//
// Manhattan and Chebyshev distances are formed from coordinate differences in
// float32, coordinate 0 first (sum_t |q_t - r_t|, max_t |q_t - r_t|).  The
// Euclidean one is expanded, ||q - r||^2 = ||q||^2 + ||r||^2 - 2 q.r: one
// fused multiply-add per coordinate for the product, the squared norms summed
// from the same staged coordinates, which are taken relative to a centre c
// (the first reference of the CTA's split): q' = fl(q - c), r' = fl(r - c).
// What the selection ranks is a LOWER BOUND of the exact squared distance,
// L = (1 - g) (||q'||^2 + ||r'||^2) - 2 q'.r' with g = 4 (d + 6) 2^-24, clamped
// at 0: each norm and the product carry at most gamma_d = d u / (1 - d u)
// relative error over the sums of their terms (u = 2^-24; fused
// multiply-adds in any order), |q'.r'| summed termwise is at most
// (||q'||^2 + ||r'||^2) / 2, the last three roundings add 3 u of the same, and
// the rounding of the centred coordinates moves the distance by at most
// (4 u + O(u^2)) (||q'||^2 + ||r'||^2) (||q - r|| >= ||q' - r'|| - u (||q'|| + ||r'||)
// to first order), so the float32 L falls short of ||q - r||^2 by at least
// (g - 2 gamma_d - 7 u - O(u^2)) (||q'||^2 + ||r'||^2) >= 0.  The finalize re-ranks the
// kept candidates with exact float32 differences; a reference a split leaves
// out has L >= the split's largest kept L, so the finalize's completeness test
// on that largest key holds for the exact distances as well.
#include "knn_internal.cuh"

namespace knn {
namespace {

constexpr int kThreads = 256;
constexpr int kDK = 16;    // coordinates per shared-memory stage
constexpr int kTM = 128;   // references per tile

// CTA shapes: TY x TX threads, each an RR (queries) x CN (references)
// micro-tile whose references come in groups of G consecutive columns;
// MINB CTAs per SM (the register bound).  The 128-row shape loads 16 floats
// from shared memory per 64 distance terms (the 64-row one 12 per 32), which
// is what bounds the arithmetic at large n; the 16-row shape leaves room for
// the heaps of large c.
template <int ROWS>
struct CCShape;
template <>
struct CCShape<128> {      // 16 x 16 threads, 8 queries x 8 references each
    static constexpr int TY = 16, TX = 16, RR = 8, CN = 8, G = 4, MINB = 2;
};
template <>
struct CCShape<64> {       // 16 x 16 threads, 4 queries x 8 references each
    static constexpr int TY = 16, TX = 16, RR = 4, CN = 8, G = 4, MINB = 3;
};
template <>
struct CCShape<16> {       // 4 x 64 threads, 4 queries x 2 references each
    static constexpr int TY = 4, TX = 64, RR = 4, CN = 2, G = 2, MINB = 3;
};

// Row pitch of the finished distance tile (floats).  The selection reads it
// 16 bytes per thread with TPR = kThreads / ROWS threads per row at 16-byte
// strides; a quarter warp then spans 8 / TPR rows, and a pitch of 4 TPR
// (mod 32) banks puts them on distinct banks.
template <int ROWS>
constexpr int cc_dst() {
    return (kThreads / ROWS) <= 4 ? kTM + 4 * (kThreads / ROWS) : kTM + 4;
}

// Shared memory: the two coordinate-stage buffers (queries and references)
// and the finished distance tile use the same space, one after the other;
// the heaps follow.
template <int ROWS>
constexpr size_t cc_stage_bytes() {
    return sizeof(float) * 2 * kDK * ((ROWS + 4) + (kTM + 4));
}
template <int ROWS>
constexpr size_t cc_union_bytes() {
    return cc_stage_bytes<ROWS>() > sizeof(float) * ROWS * cc_dst<ROWS>()
               ? cc_stage_bytes<ROWS>()
               : sizeof(float) * ROWS * cc_dst<ROWS>();
}
// ... then the squared norms of the CTA's queries and of the current reference
// tile (Euclidean).
template <int ROWS>
constexpr size_t cc_smem_bytes(int c) {
    return cc_union_bytes<ROWS>() + sizeof(uint64_t) * static_cast<size_t>(c) * ROWS +
           sizeof(float) * (ROWS + kTM);
}

// Max-heap (largest key at slot 0) of c keys, slot-major with stride ROWS.
// Place `key` at slot i, whose subtrees are heaps, and sift it down.
template <int ROWS>
__device__ __forceinline__ void heap_sift_down(uint64_t* h, int c, int i, uint64_t key) {
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
// Replace the top by `key` (key < top).
template <int ROWS>
__device__ __forceinline__ void heap_replace_top(uint64_t* h, int c, uint64_t key) {
    heap_sift_down<ROWS>(h, c, 0, key);
}
// Make slots 0..c-1 (any order) a heap (Floyd's bottom-up construction).
template <int ROWS>
__device__ __forceinline__ void heapify(uint64_t* h, int c) {
    for (int i = c / 2 - 1; i >= 0; --i) heap_sift_down<ROWS>(h, c, i, h[i * ROWS]);
}

// Two float32 lanes: acc + (a, a) * (b0, b1), one query coordinate times the
// same coordinate of two references, one rounding per lane.
__device__ __forceinline__ uint64_t dot_pair(float a, float b0, float b1, uint64_t acc) {
    uint64_t r;
    asm("{\n .reg .b64 x, y;\n mov.b64 x, {%1, %1};\n mov.b64 y, {%2, %3};\n"
        " fma.rn.f32x2 %0, x, y, %4;\n}"
        : "=l"(r) : "f"(a), "f"(b0), "f"(b1), "l"(acc));
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
// the selection has consumed them (two more barriers per tile).
// Euclidean products run as two-lane float32 fused multiply-adds; the
// threads below kTM (below ROWS, in a CTA's first tile) also sum the squares
// of reference (query) tid's staged coordinates, its squared norm.
template <int METRIC, int ROWS>
__global__ void __launch_bounds__(kThreads, CCShape<ROWS>::MINB)
cc_select_kernel(const float* __restrict__ Q, int64_t n, const float* __restrict__ R,
                 int64_t m, int32_t d, CandidateSet cand) {
    using S = CCShape<ROWS>;
    static_assert(S::TY * S::TX == kThreads, "thread shape");
    static_assert(S::TY * S::RR == ROWS && S::TX * S::CN == kTM, "tile shape");
    static_assert(S::CN % 2 == 0 && S::G % 2 == 0 && S::RR % 4 == 0, "column pairs, row quads");
    constexpr int QST = ROWS + 4;      // padded strides (bank spread)
    constexpr int RST = kTM + 4;
    constexpr int DST = cc_dst<ROWS>();
    constexpr int TPR = kThreads / ROWS;         // selection threads per query row
    constexpr int VPT = kTM / (4 * TPR);         // float4s of the tile per selection thread
    static_assert(TPR <= 32 && 32 % TPR == 0 && VPT * 4 <= 64, "selection shape");
    constexpr int QPT = ROWS * kDK / kThreads;   // query values per thread and step
    constexpr int RPT = kTM * kDK / kThreads;    // reference values per thread and step
    constexpr int CP = S::CN / 2;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Qs = reinterpret_cast<float*>(smem_raw);            // [2][kDK][QST]
    float* Rs = Qs + 2 * kDK * QST;                            // [2][kDK][RST]
    float* Dt = reinterpret_cast<float*>(smem_raw);            // [ROWS][DST], over the stages
    uint64_t* heap = reinterpret_cast<uint64_t*>(smem_raw + cc_union_bytes<ROWS>());  // [c][ROWS]
    float* nqs = reinterpret_cast<float*>(heap + static_cast<size_t>(cand.c) * ROWS);   // [ROWS]
    float* nrs = nqs + ROWS;                                                             // [kTM]
    float nq_acc = 0.f, nr_acc = 0.f;   // squared norm of query / reference tid (Euclidean)
    const float g1 = 1.f - 4.f * static_cast<float>(d + 6) * 5.9604644775390625e-8f;   // 1 - g

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
    // selection roles: thread tid tests row srow of a finished tile; the lane
    // with ssub == 0 (the row's leader) owns the row's heap and keeps its
    // largest key and that key's distance (+inf while the heap has room).
    // Until the heap holds c keys they are appended unordered (slots 0..fill-1)
    // and the c-th makes it a heap at once: the first tile's keys, which all
    // pass, cost one store each instead of a sift each.  The finalize reads a
    // split's keys as a set, so a heap left short (a split of fewer than c
    // references) needs no order.
    const int srow = tid / TPR, ssub = tid % TPR;
    const bool leader = ssub == 0;
    const bool srow_live = qbase + srow < n;
    uint64_t top = kEmptyKey;
    float top_d = __int_as_float(0x7f800000);
    int fill = 0;

    float pq[QPT], pr[RPT];
    // Euclidean: coordinates are staged relative to the split's first
    // reference (distances do not change; the norms, and with them the
    // slack of the lower bound, become those of the data's spread rather than
    // of its offset from the origin).  A thread's elements of a step all have
    // coordinate tid % kDK (kThreads is a multiple of kDK): one centre value,
    // loaded with them and taken off as they are stored to shared memory (so
    // the loads stay in flight during the step before).  Rows past the data
    // then hold -c instead of 0: their distances are masked anyway.
    const float* cen = R + (r_begin < m ? r_begin : 0) * static_cast<int64_t>(d);
    float pcv = 0.f;
    auto fetch = [&](int h) {
        const int64_t tbase = r_begin + static_cast<int64_t>(h / stages) * kTM;
        const int dbase = (h % stages) * kDK;
        const int ct = dbase + tid % kDK;
        pcv = (METRIC == kL2 && ct < d) ? cen[ct] : 0.f;
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
            qs[(e % kDK) * QST + e / kDK] = METRIC == kL2 ? pq[u] - pcv : pq[u];
        }
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int e = tid + u * kThreads;
            rs[(e % kDK) * RST + e / kDK] = METRIC == kL2 ? pr[u] - pcv : pr[u];
        }
        __syncthreads();
        if (h + 1 < steps) fetch(h + 1);
        if constexpr (METRIC == kL2) {
            if (tid < kTM) {
#pragma unroll
                for (int t = 0; t < kDK; ++t) nr_acc = fmaf(rs[t * RST + tid], rs[t * RST + tid], nr_acc);
            }
            if (h < stages && tid < ROWS) {
#pragma unroll
                for (int t = 0; t < kDK; ++t) nq_acc = fmaf(qs[t * QST + tid], qs[t * QST + tid], nq_acc);
            }
        }
#pragma unroll 4
        for (int t = 0; t < kDK; ++t) {
            float qv[S::RR], rv[S::CN];
#pragma unroll
            for (int i = 0; i < S::RR; i += 4) {
                const float4 q4 = *reinterpret_cast<const float4*>(&qs[t * QST + ty * S::RR + i]);
                qv[i] = q4.x; qv[i + 1] = q4.y; qv[i + 2] = q4.z; qv[i + 3] = q4.w;
            }
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
                        acc2[i][j] = dot_pair(qv[i], rv[2 * j], rv[2 * j + 1], acc2[i][j]);
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
        if constexpr (METRIC == kL2) {
            if (tid < kTM) {
                nrs[tid] = nr_acc;
                nr_acc = 0.f;
            }
            if (h == stages - 1 && tid < ROWS) nqs[tid] = nq_acc;
        }
        __syncthreads();
        // the lower bound of the squared distance from the product and the norms
        auto lower = [g1](float nq, float nr, float dot) {
            return fmaxf(0.f, fmaf(-2.f, dot, g1 * (nq + nr)));
        };
#pragma unroll
        for (int i = 0; i < S::RR; ++i) {
            float* drow = Dt + (ty * S::RR + i) * DST;
            const float nq = METRIC == kL2 ? nqs[ty * S::RR + i] : 0.f;
#pragma unroll
            for (int g = 0; g < S::CN / S::G; ++g) {
                const int col = g * (S::TX * S::G) + tx * S::G;
                if constexpr (METRIC == kL2) {
                    const uint64_t p0 = acc2[i][g * S::G / 2];
                    const uint64_t p1 = acc2[i][(g * S::G / 2 + 1) % CP];
                    if constexpr (S::G == 4) {
                        const float4 nr = *reinterpret_cast<const float4*>(nrs + col);
                        *reinterpret_cast<float4*>(drow + col) =
                            make_float4(lower(nq, nr.x, pair_lo(p0)), lower(nq, nr.y, pair_hi(p0)),
                                        lower(nq, nr.z, pair_lo(p1)), lower(nq, nr.w, pair_hi(p1)));
                    } else {
                        const float2 nr = *reinterpret_cast<const float2*>(nrs + col);
                        *reinterpret_cast<float2*>(drow + col) =
                            make_float2(lower(nq, nr.x, pair_lo(p0)), lower(nq, nr.y, pair_hi(p0)));
                    }
                } else {
                    if constexpr (S::G == 4)
                        *reinterpret_cast<float4*>(drow + col) =
                            make_float4(acc[i][g * 4], acc[i][g * 4 + 1], acc[i][g * 4 + 2], acc[i][g * 4 + 3]);
                    else
                        *reinterpret_cast<float2*>(drow + col) = make_float2(acc[i][g * 2], acc[i][g * 2 + 1]);
                }
            }
#pragma unroll
            for (int j = 0; j < S::CN; ++j) acc[i][j] = 0.f;
#pragma unroll
            for (int j = 0; j < CP; ++j) acc2[i][j] = 0ull;
        }
        __syncthreads();
        // selection.  Thread (srow, ssub) tests the float4s ssub, ssub + TPR,
        // ... of row srow against the row's current largest distance (from
        // the leader: a stale, larger value only lets more through) and sets
        // bit 4v + e of its mask for element e of its v-th float4 when it may
        // enter the heap.  The leader gathers the TPR masks and inserts.
        {
            const int cols = static_cast<int>(min(static_cast<int64_t>(kTM), r_end - tbase));
            const int lead_lane = (tid & 31) & ~(TPR - 1);
            const float thr = __shfl_sync(0xffffffffu, top_d, lead_lane);
            const float* drow = Dt + srow * DST;
            uint64_t mask = 0ull;
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const int c0 = 4 * (v * TPR + ssub);
                const float4 x = *reinterpret_cast<const float4*>(drow + c0);
                const uint32_t b = ((x.x <= thr && c0 + 0 < cols) ? 1u : 0u) |
                                   ((x.y <= thr && c0 + 1 < cols) ? 2u : 0u) |
                                   ((x.z <= thr && c0 + 2 < cols) ? 4u : 0u) |
                                   ((x.w <= thr && c0 + 3 < cols) ? 8u : 0u);
                mask |= static_cast<uint64_t>(b) << (4 * v);
            }
            if (!srow_live) mask = 0ull;
            uint64_t sub_mask[TPR];
#pragma unroll
            for (int u = 0; u < TPR; ++u) sub_mask[u] = __shfl_sync(0xffffffffu, mask, lead_lane + u);
            if (leader) {
                uint64_t* hp = heap + srow;
#pragma unroll
                for (int u = 0; u < TPR; ++u) {
                    uint64_t bits = sub_mask[u];
                    while (bits) {
                        const int b = __ffsll(static_cast<long long>(bits)) - 1;
                        bits &= bits - 1;
                        const int col = 4 * ((b >> 2) * TPR + u) + (b & 3);
                        const float v = drow[col];
                        if (fill < c) {
                            hp[fill * ROWS] = make_key(v, static_cast<uint32_t>(tbase + col));
                            if (++fill == c) {
                                heapify<ROWS>(hp, c);
                                top = hp[0];
                                top_d = key_dist(top);
                            }
                        } else if (v <= top_d) {
                            const uint64_t key = make_key(v, static_cast<uint32_t>(tbase + col));
                            if (key < top) {
                                heap_replace_top<ROWS>(hp, c, key);
                                top = hp[0];
                                top_d = key_dist(top);
                            }
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
constexpr int64_t kWideRowsMinN = 8192; // 128-row CTAs only for query sets this large

// The CTA shape (queries per CTA) for n queries and c candidates, and the
// CTAs of it one SM holds: 128 rows when n is large and their heaps leave
// room for two CTAs per SM, else 64 when the shape fits, else 16.
int cc_rows(int64_t n, int32_t c, int64_t* per_sm) {
    int rows = 16;
    size_t smem = cc_smem_bytes<16>(c);
    int minb = CCShape<16>::MINB;
    if (n >= kWideRowsMinN && 2 * (cc_smem_bytes<128>(c) + kSmemPerCta) <= kSmemPerSm) {
        rows = 128;
        smem = cc_smem_bytes<128>(c);
        minb = CCShape<128>::MINB;
    } else if (cc_smem_bytes<64>(c) <= kSmemCap) {
        rows = 64;
        smem = cc_smem_bytes<64>(c);
        minb = CCShape<64>::MINB;
    }
    int64_t k = static_cast<int64_t>(kSmemPerSm / (smem + kSmemPerCta));
    if (k > minb) k = minb;
    if (k < 1) k = 1;
    *per_sm = k;
    return rows;
}

}  // namespace

int cc_plan_splits(int64_t n, int64_t m, int32_t c, int num_sms, int max_pool,
                   int64_t* chunk_out) {
    int64_t per_sm = 1;
    const int64_t rows = cc_rows(n, c, &per_sm);
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
    // fewer than two CTAs per SM (one per SM for the one-CTA shapes), with 5%
    // slack, at least enough splits for two are taken.
    int64_t s_min = 1;
    const int64_t want = (per_sm < 2 ? per_sm : 2) * sms;
    if (tiles * 100 < want * 95) s_min = (want + tiles - 1) / tiles;
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
    int64_t per_sm = 1;
    const int rows = cc_rows(n, cand.c, &per_sm);
    if (rows == 16 && cc_smem_bytes<16>(cand.c) > kSmemCap) return cudaErrorInvalidValue;
    if (launches) ++*launches;
    if (metric == kL2)
        return rows == 128 ? launch_rows<kL2, 128>(Q, n, R, m, d, cand, st)
               : rows == 64 ? launch_rows<kL2, 64>(Q, n, R, m, d, cand, st)
                            : launch_rows<kL2, 16>(Q, n, R, m, d, cand, st);
    if (metric == kL1)
        return rows == 128 ? launch_rows<kL1, 128>(Q, n, R, m, d, cand, st)
               : rows == 64 ? launch_rows<kL1, 64>(Q, n, R, m, d, cand, st)
                            : launch_rows<kL1, 16>(Q, n, R, m, d, cand, st);
    return rows == 128 ? launch_rows<kLinf, 128>(Q, n, R, m, d, cand, st)
           : rows == 64 ? launch_rows<kLinf, 64>(Q, n, R, m, d, cand, st)
                        : launch_rows<kLinf, 16>(Q, n, R, m, d, cand, st);
}

}  // namespace knn
