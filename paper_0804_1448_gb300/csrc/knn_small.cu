// knn_small.cu -- float32 select for small reference sets: every distance of
// a query held in shared memory and the c smallest found by an exact
// selection, with no data-dependent serial work.
//
// Steps 1-3 of the brute-force algorithm of Sec. 2.1 for the eight queries of
// a CTA (their rows staged in shared memory): the references go by in tiles of
// 512 rows, each thread owning two rows of a tile, which it reads 16
// coordinates at a time straight into registers (the next step's loads in
// flight while one is used) and accumulates their float32 distances to all
// eight queries at once (coordinate differences; Euclidean two coordinates to
// an instruction, as even and odd partial sums added at the end; the float32
// rounding bound the later stages use holds for any order of the additions),
// and writes them to the queries' rows of m distances in shared memory.  Then each warp selects for its query: the c-th
// smallest distance is found by a bisection over the order-preserving bit
// patterns (each step a warp-wide count over distances held in registers) or,
// for rows longer than 48 per lane, by a radix selection of 8 bits per pass
// over the row in shared memory (a per-warp histogram per pass), and the keys
// below it, plus the lowest-index ones equal to it, are compacted in index
// order by ballots.  The output is a candidate set with one split per query of
// at least the c nearest keys (a few spare slots let the bisection stop at the
// first midpoint whose count fits them; unused slots are empty), the
// finalize's float32 input.
//
// For reference sets of a few thousand points the heap-based select spends
// its time in the first tiles, where almost every distance enters the heap
// one after another in divergent code; here every step is the same for all
// lanes.
#include "knn_internal.cuh"

namespace knn {
namespace {

constexpr int kWarps = 8;                 // queries per CTA
constexpr int kThreads = 32 * kWarps;
constexpr int kRowsPerThread = 2;         // reference rows of a tile per thread
constexpr int kTileRefs = kRowsPerThread * kThreads;   // references per tile
constexpr int kChunk = 16;                // coordinates per step

template <int METRIC>
__device__ __forceinline__ float term(float acc, float diff) {
    if (METRIC == kL2) return fmaf(diff, diff, acc);
    if (METRIC == kL1) return acc + fabsf(diff);
    return fmaxf(acc, fabsf(diff));
}

// acc + (y - x)^2 on two float32 lanes, y and x each a pair of consecutive
// coordinates as one 64-bit register (as loaded): one two-lane subtraction and
// one two-lane fused multiply-add, rounded per lane as the scalar subf / fmaf
// pair would be.
__device__ __forceinline__ uint64_t sq_step2(uint64_t acc, uint64_t y, uint64_t x) {
    uint64_t r;
    asm("{\n .reg .b64 t;\n sub.rn.f32x2 t, %2, %3;\n fma.rn.f32x2 %0, t, t, %1;\n}"
        : "=l"(r) : "l"(acc), "l"(y), "l"(x));
    return r;
}
__device__ __forceinline__ float lo_f(uint64_t v) { return __uint_as_float(static_cast<uint32_t>(v)); }
__device__ __forceinline__ float hi_f(uint64_t v) { return __uint_as_float(static_cast<uint32_t>(v >> 32)); }

// One thread's distances from its kRowsPerThread reference rows to the CTA's
// queries: Euclidean as a pair of partial sums (even and odd coordinates),
// the other metrics as one scalar.  Four coordinates travel as two 64-bit
// pairs (ulonglong2), so the two-lane instructions take them as loaded.
template <int METRIC>
struct RowAcc {
    uint64_t e[kRowsPerThread][kWarps];
    float s[kRowsPerThread][kWarps];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int r = 0; r < kRowsPerThread; ++r)
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                e[r][w] = 0ull;
                s[r][w] = 0.f;
            }
    }
    // four coordinates x[r] of each of the thread's rows against the same
    // four of every query row (q: kWarps rows, pitch qv 16-byte units)
    __device__ __forceinline__ void add(const ulonglong2 (&x)[kRowsPerThread], const ulonglong2* q, int qv) {
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const ulonglong2 y = q[w * qv];
#pragma unroll
            for (int r = 0; r < kRowsPerThread; ++r) {
                if constexpr (METRIC == kL2) {
                    e[r][w] = sq_step2(e[r][w], y.x, x[r].x);
                    e[r][w] = sq_step2(e[r][w], y.y, x[r].y);
                } else {
                    float a = s[r][w];
                    a = term<METRIC>(a, lo_f(y.x) - lo_f(x[r].x));
                    a = term<METRIC>(a, hi_f(y.x) - hi_f(x[r].x));
                    a = term<METRIC>(a, lo_f(y.y) - lo_f(x[r].y));
                    a = term<METRIC>(a, hi_f(y.y) - hi_f(x[r].y));
                    s[r][w] = a;
                }
            }
        }
    }
    __device__ __forceinline__ float result(int r, int w) const {
        if constexpr (METRIC == kL2) return lo_f(e[r][w]) + hi_f(e[r][w]);
        return s[r][w];
    }
};

// PER: distances per lane held in registers for the selection (m <= 32 PER);
// 0: the selection reads them from shared memory.
// c_need: the fewest keys a query keeps (its c nearest); cand.c >= c_need
// slots, the spare ones let the bisection stop early.
template <int METRIC, int PER>
__global__ void __launch_bounds__(kThreads, 2)
small_select_kernel(const float* __restrict__ Q, int64_t n, const float* __restrict__ R,
                    int32_t m, int32_t d, int32_t c_need, CandidateSet cand) {
    extern __shared__ __align__(16) float sm[];
    const int pq = (d + kChunk - 1) / kChunk * kChunk;   // query pitch: whole chunks, zero padded
    float* Qw = sm;                                       // [kWarps][pq]
    float* Dw = Qw + kWarps * pq;                         // [kWarps][m]
    int* Hw = reinterpret_cast<int*>(Dw + static_cast<size_t>(kWarps) * m);   // [kWarps][256]
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t q = static_cast<int64_t>(blockIdx.x) * kWarps + warp;
    const bool live = q < n;
    float* drow = Dw + static_cast<size_t>(warp) * m;
    for (int i = threadIdx.x; i < kWarps * pq; i += kThreads) {
        const int w = i / pq, t = i % pq;
        const int64_t qq = static_cast<int64_t>(blockIdx.x) * kWarps + w;
        Qw[i] = (qq < n && t < d) ? Q[qq * d + t] : 0.f;
    }
    const int nch = pq / kChunk;
    const int ntiles = (m + kTileRefs - 1) / kTileRefs;
    const int steps = ntiles * nch;
    // step s = (tile s / nch, chunk s % nch): each thread owns rows
    // tile * kTileRefs + r * kThreads + threadIdx.x (r < kRowsPerThread) of
    // every tile and is their only reader, so their chunks go straight from
    // global memory into registers (zeros beyond the rows and coordinates;
    // 16-byte loads when rows are whole float4s, d % 4 == 0 and R 16-byte
    // aligned), the next step's loads issued before the current step is used
    const bool vec = (d & 3) == 0 && (reinterpret_cast<uintptr_t>(R) & 15) == 0;
    const int me = threadIdx.x;
    auto pack = [](float a, float b) {
        return static_cast<uint64_t>(__float_as_uint(a)) | (static_cast<uint64_t>(__float_as_uint(b)) << 32);
    };
    // x[g][r]: coordinates 4g..4g+3 of the chunk of row r
    auto load = [&](ulonglong2 (&x)[kChunk / 4][kRowsPerThread], int tile, int ch) {
        const int c0 = ch * kChunk;
#pragma unroll
        for (int r = 0; r < kRowsPerThread; ++r) {
            const int64_t row = static_cast<int64_t>(tile) * kTileRefs + r * kThreads + me;
            const bool rok = row < m;
            const float* src = R + (rok ? row : 0) * d + c0;
#pragma unroll
            for (int g = 0; g < kChunk / 4; ++g) {
                if (vec) {
                    x[g][r] = (rok && c0 + 4 * g < d) ? __ldg(reinterpret_cast<const ulonglong2*>(src + 4 * g))
                                                      : make_ulonglong2(0ull, 0ull);
                } else {
                    const int t = c0 + 4 * g;
                    x[g][r].x = pack((rok && t < d) ? __ldg(src + 4 * g) : 0.f,
                                     (rok && t + 1 < d) ? __ldg(src + 4 * g + 1) : 0.f);
                    x[g][r].y = pack((rok && t + 2 < d) ? __ldg(src + 4 * g + 2) : 0.f,
                                     (rok && t + 3 < d) ? __ldg(src + 4 * g + 3) : 0.f);
                }
            }
        }
    };
    // (tile, chunk) of the step computed next and of the step loaded next
    int ct = 0, cc = 0, lt = 0, lc = 0;
    auto advance = [nch](int& t, int& c) {
        if (++c == nch) {
            c = 0;
            ++t;
        }
    };
    RowAcc<METRIC> acc;
    acc.clear();
    ulonglong2 xb[2][kChunk / 4][kRowsPerThread];
    if (steps > 0) {
        load(xb[0], lt, lc);
        advance(lt, lc);
    }
    __syncthreads();               // the query rows are staged
    for (int st0 = 0; st0 < steps; st0 += 2) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int st = st0 + u;
            if (st < steps) {
                // buffer (u + 1) % 2 was used by step st - 1
                if (st + 1 < steps) {
                    load(xb[(u + 1) % 2], lt, lc);
                    advance(lt, lc);
                }
                const ulonglong2* q2 = reinterpret_cast<const ulonglong2*>(Qw) + cc * (kChunk / 4);
#pragma unroll
                for (int g = 0; g < kChunk / 4; ++g) acc.add(xb[u][g], q2 + g, pq / 4);
                if (cc == nch - 1) {
#pragma unroll
                    for (int r = 0; r < kRowsPerThread; ++r) {
                        const int row = ct * kTileRefs + r * kThreads + me;
                        if (row < m) {
#pragma unroll
                            for (int w = 0; w < kWarps; ++w)
                                Dw[static_cast<size_t>(w) * m + row] = acc.result(r, w);
                        }
                    }
                    acc.clear();
                }
                advance(ct, cc);
            }
        }
    }
    __syncthreads();               // every row of Dw is written
    __syncwarp();
    if (!live) return;   // no block-wide barrier follows

    // distances are >= 0: their bit patterns order like the values.  PER > 0:
    // the lane's (j = lane + 32 i) go to registers, absent ones as all-ones,
    // which no count below reaches; PER == 0: every pass reads the row from
    // shared memory (long rows, which would not fit the registers)
    const unsigned full = 0xffffffffu;
    uint32_t v[PER > 0 ? PER : 1];
    if constexpr (PER > 0) {
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int j = lane + 32 * i;
            v[i] = j < m ? __float_as_uint(drow[j]) : 0xffffffffu;
        }
    }
    // the lane's count of patterns u with pred(u), over its j = lane + 32 i < m
    auto count_if = [&](auto&& pred) {
        int c = 0;
        if constexpr (PER > 0) {
#pragma unroll
            for (int i = 0; i < PER; ++i) c += pred(v[i]) ? 1 : 0;
        } else {
#pragma unroll 4
            for (int j = lane; j < m; j += 32) c += pred(__float_as_uint(drow[j])) ? 1 : 0;
        }
        return static_cast<int>(__reduce_add_sync(full, static_cast<unsigned>(c)));
    };
    uint32_t lo = 0xffffffffu, hi = 0u;
    if constexpr (PER > 0) {
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            lo = min(lo, v[i]);
            if (lane + 32 * i < m) hi = max(hi, v[i]);
        }
    } else {
        for (int j = lane; j < m; j += 32) {
            const uint32_t u = __float_as_uint(drow[j]);
            lo = min(lo, u);
            hi = max(hi, u);
        }
    }
    lo = __reduce_min_sync(full, lo);
    hi = __reduce_max_sync(full, hi);
    const int slots = cand.c;
    // tau: a pattern with c_need <= count(<= tau), either one whose count also
    // fits the slots or the smallest pattern reaching c_need
    uint32_t tau;
    int cnt_b;
    if constexpr (PER > 0) {
        // bisection from [lo, hi] (count(<= hi) = m >= c_need), each step one
        // count over the registers; it stops at the first midpoint whose count
        // fits the slots
        uint32_t a = lo, b = hi;
        cnt_b = m;
        while (a < b && cnt_b > slots) {
            const uint32_t mid = a + (b - a) / 2;
            const int cnt = count_if([mid](uint32_t u) { return u <= mid; });
            if (cnt >= c_need) {
                b = mid;
                cnt_b = cnt;
            } else {
                a = mid + 1;
            }
        }
        tau = b;
    } else {
        // radix selection, 8 bits per pass from the highest bit in which lo
        // and hi differ (the bits above it are common to the whole row): a
        // histogram of the digit over the patterns that share the prefix fixed
        // so far picks the digit holding the c_need-th smallest; it stops once
        // everything up to the end of that digit's range fits the slots
        tau = lo;
        if (lo != hi) {
            int* hist = Hw + warp * 256;
            const int hb = 31 - __clz(lo ^ hi);
            int sh = hb >= 7 ? hb - 7 : 0;
            uint32_t hmask = sh + 8 >= 32 ? 0u : (0xffffffffu << (sh + 8));
            uint32_t prefix = lo & hmask;
            int before = 0;   // patterns below the prefix's range
            while (true) {
                for (int i = lane; i < 256; i += 32) hist[i] = 0;
                __syncwarp();
                for (int j = lane; j < m; j += 32) {
                    const uint32_t u = __float_as_uint(drow[j]);
                    if ((u & hmask) == prefix) atomicAdd(&hist[(u >> sh) & 255u], 1);
                }
                __syncwarp();
                // eight bins per lane; the lane whose bins hold the c_need-th
                // pattern finds its digit, the count before it and in it
                const int4 h0 = reinterpret_cast<const int4*>(hist)[2 * lane];
                const int4 h1 = reinterpret_cast<const int4*>(hist)[2 * lane + 1];
                const int h[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
                int s8 = 0;
#pragma unroll
                for (int i = 0; i < 8; ++i) s8 += h[i];
                int incl = s8;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v2 = __shfl_up_sync(full, incl, o);
                    if (lane >= o) incl += v2;
                }
                const int excl = incl - s8;
                const bool mine = before + excl < c_need && c_need <= before + incl;
                int digit = 0, cb = 0, cin = 0;
                if (mine) {
                    int run = excl;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        if (before + run + h[i] >= c_need && cin == 0) {
                            digit = 8 * lane + i;
                            cb = run;
                            cin = h[i];
                        }
                        run += h[i];
                    }
                }
                const int owner = __ffs(__ballot_sync(full, mine)) - 1;
                digit = __shfl_sync(full, digit, owner);
                cb = __shfl_sync(full, cb, owner);
                cin = __shfl_sync(full, cin, owner);
                prefix = (prefix & hmask) | (static_cast<uint32_t>(digit) << sh);
                if (before + cb + cin <= slots || sh == 0) {
                    tau = prefix | (sh ? ((1u << sh) - 1u) : 0u);
                    break;
                }
                before += cb;
                hmask = 0xffffffffu << sh;
                sh = sh >= 8 ? sh - 8 : 0;
                __syncwarp();      // every lane has read the histogram
            }
        }
        cnt_b = count_if([tau](uint32_t u) { return u <= tau; });
    }
    const int below = count_if([tau](uint32_t u) { return u < tau; });
    // every key below tau, then keys equal to it, lowest indices first, up to
    // the slots: a key left out is never below one kept
    const int need_eq = min(cnt_b, slots) - below;
    uint64_t* out = cand.keys + (q * cand.S) * slots;
    const unsigned lt_mask = (1u << lane) - 1u;
    int pos = 0, eq_seen = 0;
    auto compact = [&](int j, uint32_t u) {
        const bool eq = j < m && u == tau;
        const unsigned beq = __ballot_sync(full, eq);
        const bool take = (j < m && u < tau) || (eq && eq_seen + __popc(beq & lt_mask) < need_eq);
        const unsigned bt = __ballot_sync(full, take);
        if (take) out[pos + __popc(bt & lt_mask)] = make_key(__uint_as_float(u), static_cast<uint32_t>(j));
        pos += __popc(bt);
        eq_seen += __popc(beq);
    };
    if constexpr (PER > 0) {
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            if (32 * i >= m) break;
            compact(lane + 32 * i, v[i]);
        }
    } else {
        for (int j0 = 0; j0 < m; j0 += 32) {
            const int j = j0 + lane;
            compact(j, j < m ? __float_as_uint(drow[j]) : 0xffffffffu);
        }
    }
    for (int e = pos + lane; e < slots; e += 32) out[e] = kEmptyKey;
}

template <int METRIC, int PER>
cudaError_t launch_per(const float* Q, int64_t n, const float* R, int64_t m, int32_t d,
                       int32_t c_need, const CandidateSet& cand, size_t smem, cudaStream_t st) {
    cudaError_t err = allow_smem<small_select_kernel<METRIC, PER>>(smem);
    if (err != cudaSuccess) return err;
    const unsigned grid = static_cast<unsigned>((n + kWarps - 1) / kWarps);
    small_select_kernel<METRIC, PER><<<grid, kThreads, smem, st>>>(Q, n, R, static_cast<int32_t>(m),
                                                                   d, c_need, cand);
    return cudaGetLastError();
}

template <int METRIC>
cudaError_t launch_metric(const float* Q, int64_t n, const float* R, int64_t m, int32_t d,
                          int32_t c_need, const CandidateSet& cand, size_t smem, cudaStream_t st) {
    if (m <= 32 * 16) return launch_per<METRIC, 16>(Q, n, R, m, d, c_need, cand, smem, st);
    if (m <= 32 * 32) return launch_per<METRIC, 32>(Q, n, R, m, d, c_need, cand, smem, st);
    if (m <= 32 * 48) return launch_per<METRIC, 48>(Q, n, R, m, d, c_need, cand, smem, st);
    return launch_per<METRIC, 0>(Q, n, R, m, d, c_need, cand, smem, st);
}

}  // namespace

size_t small_select_smem(int64_t m, int32_t d) {
    const size_t pq = (static_cast<size_t>(d) + kChunk - 1) / kChunk * kChunk;
    return sizeof(float) * (kWarps * pq + kWarps * static_cast<size_t>(m) + kWarps * 256);
}

bool small_select_fits(int64_t m, int32_t d) {
    return m >= 1 && m <= kSmallSelectMaxM && small_select_smem(m, d) <= 220 * 1024;
}

cudaError_t launch_small_select(const float* Q, int64_t n, const float* R, int64_t m, int32_t d,
                                int32_t metric, int32_t c_need, const CandidateSet& cand,
                                cudaStream_t st, int* launches) {
    if (!small_select_fits(m, d) || cand.S != 1 || c_need < 1 || c_need > m || cand.c < c_need)
        return cudaErrorInvalidValue;
    const size_t smem = small_select_smem(m, d);
    if (launches) ++*launches;
    if (metric == kL2) return launch_metric<kL2>(Q, n, R, m, d, c_need, cand, smem, st);
    if (metric == kL1) return launch_metric<kL1>(Q, n, R, m, d, c_need, cand, smem, st);
    return launch_metric<kLinf>(Q, n, R, m, d, c_need, cand, smem, st);
}

}  // namespace knn
