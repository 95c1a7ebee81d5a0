// knn_tc.cu -- tensor-core (tcgen05 / TMEM / TMA) form of the fused distance +
// per-query top-c stage, for the Euclidean distance.
//
// ||q - r||^2 = ||q||^2 + ||r||^2 - 2 q.r; for a fixed query the ranking of
// the references depends only on s(q, r) = ||r||^2 - 2 q.r, so the kernel
// computes the cross term q.r on the tensor cores (bf16 or tf32 operands,
// float32 accumulation) and ranks by s; ||q||^2 is never needed here.  The
// c best references by s per query become candidates; the finalize stage
// re-ranks them with exact float32 differences (knn_finalize.cu).
//
// One CTA owns a tile of 128 queries (the MMA's M dimension, one TMEM lane per
// query) and streams the references of its split in tiles of 128 (N):
//   warp 0     TMA producer: the query tile once, then reference tiles into a
//              ring of kStages shared-memory stages (128-byte swizzle);
//   warp 1     MMA issuer: for each reference tile, kp/16 (bf16) or kp/8
//              (tf32) tcgen05.mma into one of two TMEM accumulators, then
//              tcgen05.commit to free the smem stage and publish the tile;
//   warps 2-5  epilogue: thread t of warp w owns query row 32*(w%4)+t; it
//              reads its row of the accumulator (tcgen05.ld 32x32b), releases
//              the TMEM buffer, and pushes s = ||r||^2 - 2 acc through its own
//              bounded max-heap of c candidates in shared memory.
// Every wait on an mbarrier is bounded (kTimeoutNs); on expiry the CTA sets
// the error flag, stops, drains what it issued and frees its TMEM.
#include "knn_internal.cuh"

#include <cuda.h>
#include <cuda_bf16.h>

namespace knn {
namespace {

constexpr int kBlockM = 128;        // queries per CTA (TMEM lanes)
constexpr int kBlockN = 128;        // references per MMA tile
constexpr int kAtomBytes = 128;     // swizzle width: one K block per 128 bytes
constexpr int kTileBytes = kBlockM * kAtomBytes;   // one K block of a 128-row tile
constexpr int kThreads = 192;
constexpr int kEpiThreads = 128;
constexpr uint64_t kTimeoutNs = 1000000000ull;     // 1 s per wait
constexpr int kMaxStages = 4;
constexpr size_t kSmemLimit = 232448;              // sm_100 family, per CTA

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of `bar` with the given parity.  Returns false
// when the CTA's abort flag is raised or the time limit passes.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 31) == 0) {
            if (abort_flag && *abort_flag) return false;
            if (globaltimer() - t0 > kTimeoutNs) return false;
        }
    }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = static_cast<uint64_t>((addr & 0x3ffffu) >> 4);   // start address
    d |= static_cast<uint64_t>(1) << 16;                         // leading offset (unused)
    d |= static_cast<uint64_t>(1024 >> 4) << 32;                 // stride offset
    d |= static_cast<uint64_t>(1) << 46;                         // descriptor version
    d |= static_cast<uint64_t>(2) << 61;                         // 128-byte swizzle
    return d;
}
// Instruction descriptor: f32 accumulator, K-major A and B, M x N.
__host__ __device__ constexpr uint32_t idesc(int fmt, int M, int N) {
    return (1u << 4) | (static_cast<uint32_t>(fmt) << 7) | (static_cast<uint32_t>(fmt) << 10) |
           (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}
template <int PREC>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id,
                                    uint32_t accumulate) {
    if (PREC == kBF16) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(id), "r"(accumulate));
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(id), "r"(accumulate));
    }
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Max-heap of c keys per row, slot-major (stride kEpiThreads).
__device__ __forceinline__ void heap_replace_top(uint64_t* h, int c, uint64_t key) {
    int i = 0;
    while (true) {
        const int l = 2 * i + 1;
        if (l >= c) break;
        uint64_t big = h[l * kEpiThreads];
        int bi = l;
        if (l + 1 < c) {
            const uint64_t rv = h[(l + 1) * kEpiThreads];
            if (rv > big) { big = rv; bi = l + 1; }
        }
        if (big <= key) break;
        h[i * kEpiThreads] = big;
        i = bi;
    }
    h[i * kEpiThreads] = key;
}

struct TcShape {
    int kb;       // K blocks of 128 bytes
    int ksteps;   // MMA instructions per tile (32 bytes of K each)
    int stages;
    size_t smem;  // dynamic shared memory, including 1 KB alignment slack
};

__host__ __device__ inline size_t tc_smem_bytes(int kb, int stages, int c) {
    return 1024 + static_cast<size_t>(kb) * kTileBytes * (1 + stages) +
           static_cast<size_t>(c) * kEpiThreads * 8 + 256;
}

TcShape tc_shape(int kp, int prec, int c) {
    TcShape s;
    const int elt = (prec == kBF16) ? 2 : 4;
    s.kb = (kp * elt + kAtomBytes - 1) / kAtomBytes;
    s.ksteps = kp * elt / 32;
    s.stages = 0;
    s.smem = 0;
    for (int st = kMaxStages; st >= 2; --st) {
        if (tc_smem_bytes(s.kb, st, c) <= kSmemLimit) {
            s.stages = st;
            s.smem = tc_smem_bytes(s.kb, st, c);
            break;
        }
    }
    return s;
}

struct TcArgs {
    const float* r_norms;    // padded to a multiple of kBlockN, zero beyond m
    int64_t n, m;
    int32_t kb, ksteps, stages;
    CandidateSet cand;
    int32_t* error_flag;
};

template <int PREC>
__global__ void __launch_bounds__(kThreads, 1)
tc_select_kernel(const __grid_constant__ CUtensorMap tmap_q,
                 const __grid_constant__ CUtensorMap tmap_r, TcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);   // 1 KB aligned

    const int KB = a.kb, NST = a.stages, c = a.cand.c;
    unsigned char* sA = smem;
    unsigned char* sB = sA + KB * kTileBytes;
    uint64_t* heap = reinterpret_cast<uint64_t*>(sB + static_cast<size_t>(NST) * KB * kTileBytes);
    uint64_t* bars = heap + static_cast<size_t>(c) * kEpiThreads;
    uint64_t* full = bars;                 // [NST]  TMA -> MMA
    uint64_t* empty = bars + kMaxStages;   // [NST]  MMA -> TMA
    uint64_t* a_full = bars + 2 * kMaxStages;
    uint64_t* t_full = a_full + 1;         // [2]    MMA -> epilogue
    uint64_t* t_empty = t_full + 2;        // [2]    epilogue -> MMA
    uint64_t* drain = t_empty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t q0 = static_cast<int64_t>(blockIdx.x) * kBlockM;
    const int split = blockIdx.y;
    const int64_t r_begin = static_cast<int64_t>(split) * a.cand.chunk;
    const int64_t r_end = min(a.m, r_begin + a.cand.chunk);
    const int ntiles = static_cast<int>((r_end - r_begin + kBlockN - 1) / kBlockN);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(a_full, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&t_full[b], 1);
            mbar_init(&t_empty[b], kEpiThreads);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {   // allocate 256 TMEM columns: two 128-column accumulators
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (int e = threadIdx.x - 64; e >= 0 && e < c * kEpiThreads; e += kEpiThreads)
        heap[e] = kEmptyKey;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    auto fail = [&]() {
        *abort_flag = 1;
        atomicExch(a.error_flag, 1);
    };

    if (warp == 0) {
        // ------------------------------------------------------ TMA producer
        if (lane == 0) {
            const int box_x = kAtomBytes / ((PREC == kBF16) ? 2 : 4);
            mbar_expect_tx(a_full, KB * kTileBytes);
            for (int kb = 0; kb < KB; ++kb)
                tma_load_2d(sA + kb * kTileBytes, &tmap_q, a_full, kb * box_x,
                            static_cast<int>(q0));
            int issued = 0;
            for (int t = 0; t < ntiles; ++t) {
                const int s = t % NST;
                if (!mbar_wait(&empty[s], ((t / NST) & 1) ^ 1, abort_flag)) { fail(); break; }
                unsigned char* dst = sB + static_cast<size_t>(s) * KB * kTileBytes;
                mbar_expect_tx(&full[s], KB * kTileBytes);
                const int y = static_cast<int>(r_begin + static_cast<int64_t>(t) * kBlockN);
                for (int kb = 0; kb < KB; ++kb)
                    tma_load_2d(dst + kb * kTileBytes, &tmap_r, &full[s], kb * box_x, y);
                issued = t + 1;
            }
            // drain: every issued load has landed before the CTA may exit
            mbar_wait(a_full, 0, nullptr);
            for (int t = (issued > NST ? issued - NST : 0); t < issued; ++t)
                mbar_wait(&full[t % NST], (t / NST) & 1, nullptr);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t id = idesc(PREC == kBF16 ? 1 : 2, kBlockM, kBlockN);
            bool ok = mbar_wait(a_full, 0, abort_flag);
            if (!ok) fail();
            const uint32_t a_base = smem_u32(sA);
            for (int t = 0; ok && t < ntiles; ++t) {
                const int s = t % NST, acc = t & 1;
                if (!mbar_wait(&t_empty[acc], ((t >> 1) & 1) ^ 1, abort_flag)) { fail(); break; }
                if (!mbar_wait(&full[s], (t / NST) & 1, abort_flag)) { fail(); break; }
                tc_fence_after();
                const uint32_t b_base = smem_u32(sB + static_cast<size_t>(s) * KB * kTileBytes);
                const uint32_t d_tmem = tmem + acc * kBlockN;
                for (int ks = 0; ks < a.ksteps; ++ks) {
                    const uint32_t off = (ks >> 2) * kTileBytes + (ks & 3) * 32;
                    mma<PREC>(d_tmem, sdesc(a_base + off), sdesc(b_base + off), id, ks > 0 ? 1u : 0u);
                }
                tc_commit(&empty[s]);
                tc_commit(&t_full[acc]);
            }
            tc_commit(drain);                   // completes when every MMA above has
            mbar_wait(drain, 0, nullptr);
        }
    } else {
        // --------------------------------------------------------- epilogue
        const int quarter = warp & 3;           // TMEM lanes this warp may read
        const int row = quarter * 32 + lane;
        const int64_t q = q0 + row;
        const bool active = q < a.n;
        uint64_t* h = heap + row;
        uint64_t top = kEmptyKey;
        float thr = __int_as_float(0x7f800000);
        const uint32_t lane_addr = tmem + (static_cast<uint32_t>(quarter * 32) << 16);
        for (int t = 0; t < ntiles; ++t) {
            const int acc = t & 1;
            const bool ok = mbar_wait(&t_full[acc], (t >> 1) & 1, abort_flag);
            if (!__all_sync(0xffffffffu, ok)) { fail(); break; }   // warp-uniform exit
            tc_fence_after();
            const int64_t jbase = r_begin + static_cast<int64_t>(t) * kBlockN;
#pragma unroll 1
            for (int ch = 0; ch < kBlockN / 32; ++ch) {
                float v[32];
                __syncwarp();                   // tcgen05.ld is .sync.aligned
                tmem_ld32(lane_addr + acc * kBlockN + ch * 32, v);
                if (ch == kBlockN / 32 - 1) {
                    tc_fence_before();
                    mbar_arrive(&t_empty[acc]);
                }
                if (!active) continue;
                const int64_t j0 = jbase + ch * 32;
                const float4* nr4 = reinterpret_cast<const float4*>(a.r_norms + j0);
                const int lim = static_cast<int>(min(static_cast<int64_t>(32), r_end - j0));
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                    const float4 nr = __ldg(nr4 + g);
                    const float nv[4] = {nr.x, nr.y, nr.z, nr.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int i = g * 4 + u;
                        const float sc = fmaf(-2.f, v[i], nv[u]);
                        if (sc < thr && i < lim) {
                            heap_replace_top(h, c, make_key(sc, static_cast<uint32_t>(j0 + i)));
                            top = h[0];
                            thr = (top == kEmptyKey) ? __int_as_float(0x7f800000) : key_dist(top);
                        }
                    }
                }
            }
        }
        if (active) {
            uint64_t* out = a.cand.keys + (q * a.cand.S + split) * static_cast<int64_t>(c);
            for (int s = 0; s < c; ++s) out[s] = h[s * kEpiThreads];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
    }
}

// --------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 2-D map over a rows x kp operand: box = (128 bytes of K) x 128 rows,
// 128-byte swizzle, zero fill outside the tensor.
bool make_map(CUtensorMap* map, const void* base, int64_t rows, int kp, int prec) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const int elt = (prec == kBF16) ? 2 : 4;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(kp), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(kp) * elt};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kAtomBytes / elt), static_cast<cuuint32_t>(kBlockM)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, prec == kBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                    2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// One thread per (row, padded column): low-precision copy, zero beyond d.
template <int PREC>
__global__ void prepare_lowp_kernel(const float* __restrict__ X, int64_t rows, int32_t d,
                                    int32_t kp, void* __restrict__ out) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= rows * kp) return;
    const int64_t r = e / kp;
    const int t = static_cast<int>(e % kp);
    const float v = (t < d) ? X[r * d + t] : 0.f;
    if (PREC == kBF16) {
        reinterpret_cast<__nv_bfloat16*>(out)[e] = __float2bfloat16_rn(v);
    } else {
        uint32_t b;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(b) : "f"(v));
        reinterpret_cast<uint32_t*>(out)[e] = b;
    }
}

// One warp per row: squared norm in float32.
__global__ void norms_kernel(const float* __restrict__ X, int64_t rows, int32_t d,
                             float* __restrict__ norms) {
    const int64_t r = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (r >= rows) return;
    float acc = 0.f;
    for (int t = lane; t < d; t += 32) {
        const float v = X[r * d + t];
        acc = fmaf(v, v, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) norms[r] = acc;
}

}  // namespace

int tc_padded_dim(int32_t d, int prec) {
    const int step = (prec == kBF16) ? 16 : 8;   // 32 bytes: one MMA K step
    return (d + step - 1) / step * step;
}

int tc_max_candidates(int32_t kp, int prec) {
    const int elt = (prec == kBF16) ? 2 : 4;
    const int kb = (kp * elt + kAtomBytes - 1) / kAtomBytes;
    int c = 0;
    while (tc_smem_bytes(kb, 2, c + 8) <= kSmemLimit) c += 8;
    return c;
}

cudaError_t launch_prepare_lowp(const float* X, int64_t rows, int32_t d, int32_t kp, int prec,
                                void* X_lp, float* norms, cudaStream_t st, int* launches) {
    const int64_t total = rows * kp;
    const unsigned grid = static_cast<unsigned>((total + 255) / 256);
    if (prec == kBF16) prepare_lowp_kernel<kBF16><<<grid, 256, 0, st>>>(X, rows, d, kp, X_lp);
    else prepare_lowp_kernel<kTF32><<<grid, 256, 0, st>>>(X, rows, d, kp, X_lp);
    if (launches) ++*launches;
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess || !norms) return err;
    norms_kernel<<<static_cast<unsigned>((rows * 32 + 255) / 256), 256, 0, st>>>(X, rows, d, norms);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_tc_select(const void* Q_lp, int64_t n, const void* R_lp, const float* r_norms,
                             int64_t m, int32_t kp, int prec, const CandidateSet& cand,
                             int32_t* error_flag, cudaStream_t st, int* launches) {
    const TcShape sh = tc_shape(kp, prec, cand.c);
    if (sh.stages == 0) return cudaErrorInvalidValue;
    if (cand.chunk % kBlockN != 0) return cudaErrorInvalidValue;
    CUtensorMap mq, mr;
    if (!make_map(&mq, Q_lp, n, kp, prec) || !make_map(&mr, R_lp, m, kp, prec))
        return cudaErrorInvalidValue;
    TcArgs a;
    a.r_norms = r_norms;
    a.n = n;
    a.m = m;
    a.kb = sh.kb;
    a.ksteps = sh.ksteps;
    a.stages = sh.stages;
    a.cand = cand;
    a.error_flag = error_flag;
    dim3 grid(static_cast<unsigned>((n + kBlockM - 1) / kBlockM), static_cast<unsigned>(cand.S));
    cudaError_t err;
    if (prec == kBF16) {
        err = cudaFuncSetAttribute(tc_select_kernel<kBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(sh.smem));
        if (err != cudaSuccess) return err;
        tc_select_kernel<kBF16><<<grid, kThreads, sh.smem, st>>>(mq, mr, a);
    } else {
        err = cudaFuncSetAttribute(tc_select_kernel<kTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(sh.smem));
        if (err != cudaSuccess) return err;
        tc_select_kernel<kTF32><<<grid, kThreads, sh.smem, st>>>(mq, mr, a);
    }
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace knn
