// knn_batch.cu -- many independent searches in one persistent launch.
//
// A batch is a list of instances of the problem of Sec. 2.1, each with its own
// reference set, queries, dimension and k; the searches are independent (the
// brute-force algorithm's step 4 runs over queries with nothing shared).  Here
// the tensor-core form of every instance runs inside ONE kernel launch: one
// CTA of 576 threads per SM stays resident and pops work items from a device
// queue until it is empty.  An item is one piece of one stage of one instance:
//   0 PREP_R    rows of R  -> the augmented bf16/tf32 copy and max ||r||^2
//   1 PREP_Q    rows of Q  -> the augmented copy (and zeroed pilot maxima)
//   2 PILOT     (query tile, reference split): group maxima of sampled tiles
//   3 THRESH    queries: the per-query threshold from the pilot maxima
//   4 FILTER    (query tile, reference split): tcgen05 product, sign test,
//               hit lists
//   5 FINAL     queries: exact float32 re-rank, near-tie re-check, outputs
//   6 FALLBACK  the instance's queued queries (exact float64 pass)
// The items are queued stage by stage (every instance's stage-s items before
// any stage-(s+1) item), so an item only ever waits for items popped before
// it, which are running or done: before starting, the CTA waits until its
// instance's previous stage has completed all its items (a per-instance,
// per-stage counter).  The stages run the device code of the one-search path
// (tc_device.cuh, finalize_device.cuh), item by item; TMEM is allocated once
// per CTA and every item re-initializes (and afterwards invalidates) its
// mbarriers.
//
// Every wait is bounded: the start waits for a "ready" word that the host sets
// before the launch, and each dependency wait gives up after wait_ns, or at
// once when another CTA has raised the error flag.  A CTA that gives up raises
// the flag and leaves; the host reports KNN_ERR_TIMEOUT.  Nothing traps.
#include <algorithm>
#include <cstring>
#include <vector>

#include "finalize_device.cuh"
#include "knn_batch.cuh"
#include "tc_device.cuh"

namespace knn {
namespace {

using namespace ptx;

enum BatchStage : int32_t {
    kStPrepR = 0, kStPrepQ, kStPilot, kStThresh, kStFilter, kStFinal, kStFallback, kNumStages
};

static_assert(kNumStages == kPersistStages, "stage count");
constexpr int kBWarps = kTcThreads / 32;        // 18
constexpr int kPrepRows = kBWarps * 128;        // rows per preparation item
constexpr int kThreshQueries = kBWarps * 4;     // queries per threshold item
constexpr size_t kBatchStatic = 1536;           // static shared memory the kernel may use
constexpr size_t kBatchDyn = kSmemLimit - kBatchStatic;   // dynamic shared memory of an item

struct BatchItem {
    int32_t stage;
    int32_t inst;
    int32_t a;   // PREP: first row; PILOT / FILTER: query tile; THRESH / FINAL: first query
    int32_t b;   // PREP / THRESH / FINAL: how many; PILOT / FILTER: reference split
};

struct BatchInst {   // 64-byte aligned by its tensor maps
    CUtensorMap mq;        // the queries' low-precision copy, for TMA
    CUtensorMap mr;        // the references'
    TcArgs ta_pilot;
    TcArgs ta_filter;
    FinalizeArgs fa;
    const float* R;
    const float* Q;
    void* R_lp;
    void* Q_lp;
    uint32_t* rmax2;
    float* qscale;
    uint32_t* gmax;
    double* fb_scratch;
    int64_t m, n;
    int32_t d, kp, pilot, kbt, epi, vpl, G, cprime;
    int32_t fin_P, fin_se, fin_nv, fin_wq, fin_pw;
    int32_t prev[kNumStages];   // the stage whose completion an item of each stage waits for
    int32_t need[kNumStages];   // items of each stage
};

struct BatchDesc {
    const BatchItem* items;
    const BatchInst* insts;
    int32_t nitems;
    int32_t* head;              // next item to pop
    int32_t* done;              // [instances][kNumStages] completed items
    const int32_t* ready;       // non-zero: the host lets the kernel start
    int32_t* error_flag;        // raised by a wait that gave up (any CTA)
    uint64_t wait_ns;           // bound of every wait
    unsigned long long* stage_ns;   // [3][kNumStages]: CTA time waiting, CTA time working, items
};

__device__ __forceinline__ int32_t ld_volatile(const int32_t* p) {
    return *reinterpret_cast<const volatile int32_t*>(p);
}

// Wait until *p >= target; false when wait_ns pass or the error flag is raised.
__device__ bool wait_geq(const int32_t* p, int32_t target, const int32_t* error_flag,
                         uint64_t wait_ns) {
    if (ld_volatile(p) >= target) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        __nanosleep(128);
        if (ld_volatile(p) >= target) return true;
        if (ld_volatile(error_flag) != 0) return false;
        if (globaltimer() - t0 > wait_ns) return false;
    }
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

template <int PREC, bool PILOT, int KBT, int EPI>
__device__ __noinline__ void tc_item(const BatchInst& I, const TcArgs& ta, int64_t qtile, int split,
                                     unsigned char* smem, uint32_t tmem) {
    tc_run<PREC, PILOT, KBT, EPI, true>(&I.mq, &I.mr, ta, qtile, split, smem, tmem);
}

template <int PREC, bool PILOT, int EPI>
__device__ __forceinline__ void run_tc_item(const BatchInst& I, const TcArgs& ta, int64_t qtile,
                                            int split, unsigned char* smem, uint32_t tmem) {
    switch (I.kbt) {
        case 1: tc_item<PREC, PILOT, 1, EPI>(I, ta, qtile, split, smem, tmem); break;
        case 2: tc_item<PREC, PILOT, 2, EPI>(I, ta, qtile, split, smem, tmem); break;
        default: tc_item<PREC, PILOT, 0, EPI>(I, ta, qtile, split, smem, tmem); break;
    }
}

template <int PREC, int VPL>
__device__ __noinline__ void thresh_rows(const BatchInst& I, int64_t q0, int64_t q1, int warp,
                                            int lane) {
    for (int64_t q = q0 + warp; q < q1; q += kBWarps)
        threshold_query<PREC, VPL>(I.gmax, q, I.G, I.cprime, I.d, I.kp, I.Q_lp, I.rmax2, I.qscale,
                                   lane);
}

template <int NV>
__device__ __noinline__ void final_rows(const FinalizeArgs& fa, const BatchInst& I, int64_t q0,
                                           int64_t q1, unsigned char* smem, int warp, int lane) {
    if (warp >= I.fin_wq) return;
    unsigned char* scratch = smem + static_cast<size_t>(I.fin_pw) * warp;
    for (int64_t q = q0 + warp; q < q1; q += I.fin_wq)
        finalize_query<kL2, NV>(fa, I.fin_P, I.fin_se, q, scratch, lane);
}

// Rows [r0, r1) of R (REF) or Q into the instance's augmented low-precision
// copy, the operation of prepare_row (same arithmetic, same order), with
// kPrepInFlight rows per warp loaded before any is used: one row at a time
// leaves a warp waiting on memory for every row.  Needs d <= 128 (four
// coordinates per lane).  REF: the largest squared norm of the warp's rows is
// raised into the instance's maximum once.  QUERY: the pilot maxima rows are
// zeroed, or without a pilot the hit-code scale is set.
constexpr int kPrepInFlight = 8;

template <int PREC, bool REF>
__device__ __noinline__ void prep_rows(const BatchInst& I, int64_t r0, int64_t r1, int warp, int lane) {
    const float* X = REF ? I.R : I.Q;
    const int d = I.d, kp = I.kp;
    const size_t elt = (PREC == kBF16) ? 2 : 4;
    float nmax = 0.f;
    const int dg = d / 4;   // float4s of data per row
    if ((d & 3) == 0 && (dg == 8 || dg == 16 || dg == 32) && (reinterpret_cast<uintptr_t>(X) & 15) == 0) {
        // rows packed into the warp, 32 / dg rows per pack and lane (row
        // lane / dg, float4 lane % dg): one 16-byte load per lane and pack,
        // kPrepInFlight packs in flight, so short rows keep as many bytes in
        // flight as long ones; one 8- or 16-byte store per lane and four
        // elements, the augmentation and padding by the same lanes
        const int rpp = 32 / dg, pr = lane / dg, g0 = lane % dg, ng = kp / 4;
        const int64_t rows_per_iter = static_cast<int64_t>(rpp) * kPrepInFlight;
        for (int64_t rb = r0 + static_cast<int64_t>(warp) * rows_per_iter; rb < r1;
             rb += static_cast<int64_t>(kBWarps) * rows_per_iter) {
            float4 xv[kPrepInFlight];
#pragma unroll
            for (int u = 0; u < kPrepInFlight; ++u) {
                const int64_t r = rb + static_cast<int64_t>(u) * rpp + pr;
                xv[u] = r < r1 ? reinterpret_cast<const float4*>(X + r * d)[g0] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            float nr[kPrepInFlight];
#pragma unroll
            for (int u = 0; u < kPrepInFlight; ++u) {
                float a2 = fmaf(xv[u].x, xv[u].x, 0.f);
                a2 = fmaf(xv[u].y, xv[u].y, a2);
                a2 = fmaf(xv[u].z, xv[u].z, a2);
                nr[u] = fmaf(xv[u].w, xv[u].w, a2);
            }
            // sum over the dg lanes of each row (aligned groups of dg lanes)
            for (int o = dg / 2; o > 0; o >>= 1)
#pragma unroll
                for (int u = 0; u < kPrepInFlight; ++u) nr[u] += __shfl_xor_sync(0xffffffffu, nr[u], o);
#pragma unroll
            for (int u = 0; u < kPrepInFlight; ++u) {
                const int64_t r = rb + static_cast<int64_t>(u) * rpp + pr;
                if (r >= r1) continue;
                if (REF) nmax = fmaxf(nmax, nr[u]);
                if (!REF && g0 == 0 && !I.pilot) I.qscale[r] = hit_scale(nr[u], __uint_as_float(*I.rmax2), 0.f);
                if (!REF && I.pilot)
                    for (int g = g0; g < I.G; g += dg) I.gmax[r * I.G + g] = 0u;
                const float h = -0.5f * nr[u];
                const float hi = lowp_round<PREC>(h);
                const float lo = lowp_round<PREC>(h - hi);
                void* row = static_cast<unsigned char*>(REF ? I.R_lp : I.Q_lp) + static_cast<size_t>(r) * kp * elt;
                put4<PREC>(row, 4 * g0, xv[u]);
                for (int g = dg + g0; g < ng; g += dg) {
                    const float4 v = g == dg ? (REF ? make_float4(hi, lo, 1.f, 1.f) : make_float4(1.f, 1.f, 0.f, 0.f))
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
                    put4<PREC>(row, 4 * g, v);
                }
            }
        }
        // every lane's rows are in nmax; the warp's largest goes to the atomic
        for (int o = 16; o > 0; o >>= 1) nmax = fmaxf(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
        if (REF && lane == 0) atomicMax(I.rmax2, __float_as_uint(nmax));
        return;
    }
    for (int64_t rb = r0 + static_cast<int64_t>(warp) * kPrepInFlight; rb < r1;
         rb += static_cast<int64_t>(kBWarps) * kPrepInFlight) {
        float xv[kPrepInFlight][4];
#pragma unroll
        for (int u = 0; u < kPrepInFlight; ++u)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int t = lane + 32 * j;
                xv[u][j] = (rb + u < r1 && t < d) ? X[(rb + u) * d + t] : 0.f;
            }
        float nr[kPrepInFlight];
#pragma unroll
        for (int u = 0; u < kPrepInFlight; ++u) {
            nr[u] = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (lane + 32 * j < d) nr[u] = fmaf(xv[u][j], xv[u][j], nr[u]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int u = 0; u < kPrepInFlight; ++u) nr[u] += __shfl_xor_sync(0xffffffffu, nr[u], o);
#pragma unroll
        for (int u = 0; u < kPrepInFlight; ++u) {
            const int64_t r = rb + u;
            if (r >= r1) break;
            if (REF) nmax = fmaxf(nmax, nr[u]);
            if (!REF && lane == 0 && !I.pilot) I.qscale[r] = hit_scale(nr[u], __uint_as_float(*I.rmax2), 0.f);
            if (!REF && I.pilot)
                for (int g = lane; g < I.G; g += 32) I.gmax[r * I.G + g] = 0u;
            const float h = -0.5f * nr[u];
            const float hi = lowp_round<PREC>(h);
            const float lo = lowp_round<PREC>(h - hi);
            void* row = static_cast<unsigned char*>(REF ? I.R_lp : I.Q_lp) + static_cast<size_t>(r) * kp * elt;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int t = lane + 32 * j;
                if (t >= kp) break;
                float v = 0.f;
                if (t < d) v = xv[u][j < 4 ? j : 0];
                else if (t == d) v = REF ? hi : 1.f;
                else if (t == d + 1) v = REF ? lo : 1.f;
                else if (t == d + 2 || t == d + 3) v = REF ? 1.f : 0.f;
                put<PREC>(row, t, v);
            }
        }
    }
    if (REF && lane == 0) atomicMax(I.rmax2, __float_as_uint(nmax));
}

// The instance's queued queries, one after another, by the whole CTA.
__device__ __noinline__ void fallback_rows(const FinalizeArgs& fa, const BatchInst& I, int count,
                                           unsigned char* smem) {
    FbShared<kTcThreads>& sh = *reinterpret_cast<FbShared<kTcThreads>*>(smem);
    const FbDyn f = fb_dyn_carve(smem + align16(sizeof(FbShared<kTcThreads>)));
    for (int i = 0; i < count; ++i) fb_query<kL2, kTcThreads>(fa, fa.fallback_list[i], I.fb_scratch, sh, f);
}

template <int PREC>
__global__ void __launch_bounds__(kTcThreads, 1)
batch_kernel(const __grid_constant__ BatchDesc bd) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t s_tmem;
    __shared__ int32_t s_next, s_pre, s_abort, s_count;
    __shared__ __align__(16) TcArgs s_ta;
    __shared__ __align__(16) FinalizeArgs s_fa;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    if (warp == 1) tmem_alloc(&s_tmem, kTmemCols);
    if (threadIdx.x == 0) {
        s_abort = 0;
        if (!wait_geq(bd.ready, 1, bd.error_flag, bd.wait_ns)) {
            s_abort = 1;
            atomicExch(bd.error_flag, 1);
        }
        s_next = s_abort ? bd.nitems : atomicAdd(bd.head, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    // Shared words written by thread 0: s_next and s_abort only between the
    // last two barriers of an item (read by every thread after them); the item
    // arguments and s_pre (the item popped ahead) before the item's first
    // barrier (read after it).
    while (true) {
        const int idx = s_next;
        if (idx >= bd.nitems) break;   // CTA-uniform: s_next is stable since the last barrier
        const BatchItem it = bd.items[idx];
        const BatchInst& I = bd.insts[it.inst];
        uint64_t t_wait = 0, t_work = 0;   // thread 0: when the item's wait began and ended
        if (threadIdx.x == 0) {
            t_wait = globaltimer();
            const int ps = I.prev[it.stage];
            if (ps >= 0 && !wait_geq(&bd.done[it.inst * kNumStages + ps], I.need[ps], bd.error_flag,
                                     bd.wait_ns)) {
                s_abort = 1;
                atomicExch(bd.error_flag, 1);
            }
            // the previous stage's writes, TMA reads of them included, before this item
            __threadfence();
            fence_proxy_async();
            if (it.stage == kStPilot) s_ta = I.ta_pilot;
            if (it.stage == kStFilter) s_ta = I.ta_filter;
            if (it.stage == kStFinal || it.stage == kStFallback) s_fa = I.fa;
            if (it.stage == kStFallback) s_count = ld_volatile(I.fa.fallback_count);
            // the next item, popped now so that its latency overlaps this one
            s_pre = s_abort ? bd.nitems : atomicAdd(bd.head, 1);
            t_work = globaltimer();
        }
        __syncthreads();
        if (s_abort) break;   // CTA-uniform

        switch (it.stage) {
            case kStPrepR:
                prep_rows<PREC, true>(I, it.a, static_cast<int64_t>(it.a) + it.b, warp, lane);
                break;
            case kStPrepQ:
                prep_rows<PREC, false>(I, it.a, static_cast<int64_t>(it.a) + it.b, warp, lane);
                break;
            case kStPilot:
                run_tc_item<PREC, true, 0>(I, s_ta, it.a, it.b, smem, tmem);
                break;
            case kStThresh: {
                const int64_t q0 = it.a, q1 = static_cast<int64_t>(it.a) + it.b;
                switch (I.vpl) {
                    case 1: thresh_rows<PREC, 1>(I, q0, q1, warp, lane); break;
                    case 2: thresh_rows<PREC, 2>(I, q0, q1, warp, lane); break;
                    case 4: thresh_rows<PREC, 4>(I, q0, q1, warp, lane); break;
                    case 8: thresh_rows<PREC, 8>(I, q0, q1, warp, lane); break;
                    case 16: thresh_rows<PREC, 16>(I, q0, q1, warp, lane); break;
                    case 32: thresh_rows<PREC, 32>(I, q0, q1, warp, lane); break;
                    default: thresh_rows<PREC, 64>(I, q0, q1, warp, lane); break;
                }
                break;
            }
            case kStFilter:
                if (I.epi == 1) run_tc_item<PREC, false, 1>(I, s_ta, it.a, it.b, smem, tmem);
                else if (I.epi == 2) run_tc_item<PREC, false, 2>(I, s_ta, it.a, it.b, smem, tmem);
                else run_tc_item<PREC, false, 0>(I, s_ta, it.a, it.b, smem, tmem);
                break;
            case kStFinal: {
                const int64_t q0 = it.a, q1 = static_cast<int64_t>(it.a) + it.b;
                switch (I.fin_nv) {
                    case 1: final_rows<1>(s_fa, I, q0, q1, smem, warp, lane); break;
                    case 2: final_rows<2>(s_fa, I, q0, q1, smem, warp, lane); break;
                    case 3: final_rows<3>(s_fa, I, q0, q1, smem, warp, lane); break;
                    case 4: final_rows<4>(s_fa, I, q0, q1, smem, warp, lane); break;
                    default: final_rows<0>(s_fa, I, q0, q1, smem, warp, lane); break;
                }
                break;
            }
            case kStFallback:
                fallback_rows(s_fa, I, s_count, smem);
                break;
            default: break;
        }
        // the item's writes before its completion is counted
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            fence_proxy_async();
            atomicAdd(&bd.done[it.inst * kNumStages + it.stage], 1);
            const uint64_t t_end = globaltimer();
            atomicAdd(&bd.stage_ns[it.stage], static_cast<unsigned long long>(t_work - t_wait));
            atomicAdd(&bd.stage_ns[kNumStages + it.stage], static_cast<unsigned long long>(t_end - t_work));
            atomicAdd(&bd.stage_ns[2 * kNumStages + it.stage], 1ull);
            // another CTA gave up: stop popping
            s_next = ld_volatile(bd.error_flag) != 0 ? bd.nitems : s_pre;
        }
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

size_t persist_item_smem() { return kBatchDyn; }

// Plan every instance and lay out their buffers in a workspace of *ws_bytes
// (offsets from 0); the counters region comes first.
cudaError_t persist_plan(const std::vector<PersistInst>& in, int prec, int rerank_factor,
                         int num_sms, PersistPlan* out) {
    PersistPlan pp;
    const int ninst = static_cast<int>(in.size());
    const size_t elt = prec == kBF16 ? 2 : 4;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes, 256);
        return at;
    };
    // counters: head, done[ninst][stages], rmax2[ninst], fallback counts[ninst]; ready word
    pp.off_head = take(sizeof(int32_t));
    pp.off_done = take(sizeof(int32_t) * kNumStages * static_cast<size_t>(ninst));
    pp.off_rmax = take(sizeof(uint32_t) * static_cast<size_t>(ninst));
    pp.off_fbc = take(sizeof(int32_t) * static_cast<size_t>(ninst));
    pp.off_stage_ns = take(sizeof(unsigned long long) * 3 * kNumStages);
    pp.counters_bytes = off;
    pp.off_ready = take(sizeof(int32_t));
    pp.inst.resize(ninst);
    for (int i = 0; i < ninst; ++i) {
        const PersistInst& x = in[i];
        PersistPlan::Inst& pi = pp.inst[i];
        if (x.n == 0) continue;
        int c = rerank_factor * x.k;
        if (c > (kMaxPool - 32) / 2) c = (kMaxPool - 32) / 2;
        if (c < x.k) return cudaErrorNotSupported;
        pi.c = c;
        pi.kp = tc_padded_dim(x.d, prec);
        pi.plan = tc_plan(x.n, x.m, x.d, pi.kp, prec, c, num_sms, kBatchDyn, x.chunk);
        if (pi.plan.stages == 0) return cudaErrorNotSupported;   // rows too long for the tile
        if (x.d > 128 || pi.kp > 256) return cudaErrorNotSupported;   // the preparation's row layout
        if (x.k > kFbMaxK) return cudaErrorNotSupported;
        pi.P = (2 * c + 32 + 3) & ~3;
        if (pi.P > kMaxPool) return cudaErrorNotSupported;
        pi.pw = static_cast<int>(align16(warp_scratch_bytes(pi.P, prefix_cap(pi.P, x.k), 1, x.d, kStage)));
        pi.wq = static_cast<int>(std::min<size_t>(kBWarps, kBatchDyn / pi.pw));
        if (pi.wq < 1) return cudaErrorNotSupported;
        const size_t fb_smem = align16(sizeof(FbShared<kTcThreads>)) +
                               static_cast<size_t>(kFbCand) * (sizeof(uint64_t) + sizeof(uint32_t)) +
                               (static_cast<size_t>(x.d) + 4) * sizeof(float);
        if (fb_smem > kBatchDyn) return cudaErrorNotSupported;
        const TcPlan& p = pi.plan;
        pi.off_qlp = take(static_cast<size_t>(x.n) * pi.kp * elt);
        pi.off_rlp = take(static_cast<size_t>(x.m) * pi.kp * elt);
        if (p.pilot) pi.off_gmax = take(static_cast<size_t>(x.n) * p.G * 4);
        pi.off_lists = take(static_cast<size_t>(x.n) * p.S * p.groups * p.cap * sizeof(uint64_t));
        pi.off_counts = take(static_cast<size_t>(x.n) * p.S * p.groups * sizeof(int32_t));
        pi.off_qs = take(static_cast<size_t>(x.n) * sizeof(float));
        pi.off_list = take(static_cast<size_t>(x.n) * sizeof(int32_t));
        pi.off_scr = take(static_cast<size_t>(x.m) * sizeof(double));
    }
    pp.ws_bytes = off;
    *out = std::move(pp);
    return cudaSuccess;
}

// Build the descriptors of a planned batch whose workspace starts at ws; they
// go to device memory allocated here (out->desc, freed by persist_free).
cudaError_t persist_build(const std::vector<PersistInst>& in, const PersistPlan& pp, int prec,
                          unsigned char* ws, const PersistCounters& ctr, PersistBatch* out) {
    const int ninst = static_cast<int>(in.size());
    std::vector<BatchInst> insts(ninst);
    std::vector<std::vector<BatchItem>> by_stage(kNumStages);
    std::vector<double> work(ninst, 0.0);
    std::vector<int> order(ninst);
    for (int i = 0; i < ninst; ++i) {
        order[i] = i;
        work[i] = static_cast<double>(in[i].n) * in[i].m * in[i].d;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
    for (int oi = 0; oi < ninst; ++oi) {
        const int i = order[oi];
        const PersistInst& x = in[i];
        BatchInst& I = insts[i];
        std::memset(static_cast<void*>(&I), 0, sizeof(BatchInst));
        for (int s = 0; s < kNumStages; ++s) I.prev[s] = -1;
        if (x.n == 0) continue;
        const PersistPlan::Inst& pi = pp.inst[i];
        const TcPlan& p = pi.plan;
        I.R = x.R;
        I.Q = x.Q;
        I.m = x.m;
        I.n = x.n;
        I.d = x.d;
        I.kp = pi.kp;
        I.R_lp = ws + pi.off_rlp;
        I.Q_lp = ws + pi.off_qlp;
        I.rmax2 = reinterpret_cast<uint32_t*>(ws + pp.off_rmax) + i;
        I.qscale = reinterpret_cast<float*>(ws + pi.off_qs);
        I.gmax = p.pilot ? reinterpret_cast<uint32_t*>(ws + pi.off_gmax) : nullptr;
        I.fb_scratch = reinterpret_cast<double*>(ws + pi.off_scr);
        I.pilot = p.pilot;
        I.kbt = (p.kbs == p.kb && (p.kb == 1 || p.kb == 2)) ? p.kb : 0;
        I.epi = p.raw ? (p.pilot ? 1 : 2) : 0;
        I.G = p.G;
        I.cprime = p.cprime;
        int vpl = 1;
        while (vpl * 32 < p.G) vpl *= 2;
        I.vpl = vpl;
        if (!tc_make_map(&I.mq, I.Q_lp, x.n, pi.kp, prec, 128, 0) ||
            !tc_make_map(&I.mr, I.R_lp, x.m, pi.kp, prec, p.rb, p.kbs))
            return cudaErrorInvalidValue;
        TcArgs a{};
        a.n = x.n;
        a.m = x.m;
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
        a.error_flag = ctr.error_flag;
        I.ta_pilot = a;
        I.ta_pilot.gmax = I.gmax;
        I.ta_filter = a;
        I.ta_filter.stride = 1;
        I.ta_filter.lists = reinterpret_cast<uint64_t*>(ws + pi.off_lists);
        I.ta_filter.counts = reinterpret_cast<int32_t*>(ws + pi.off_counts);
        I.ta_filter.qscale = I.qscale;
        FinalizeArgs& fa = I.fa;
        fa.use_hits = 1;
        fa.hits.keys = I.ta_filter.lists;
        fa.hits.counts = I.ta_filter.counts;
        fa.hits.S = p.groups * p.S;
        fa.hits.cap = p.cap;
        fa.hits.c = pi.c;
        fa.cand.exact = 0;
        fa.cand.S = 1;
        fa.cand.c = pi.c;
        fa.Q = x.Q;
        fa.R = x.R;
        fa.n = x.n;
        fa.m = x.m;
        fa.d = x.d;
        fa.k = x.k;
        fa.metric = kL2;
        fa.dist_out = x.dist_out;
        fa.idx_out = x.idx_out;
        fa.fallback_count = reinterpret_cast<int32_t*>(ws + pp.off_fbc) + i;
        fa.fallback_list = reinterpret_cast<int32_t*>(ws + pi.off_list);
        fa.recheck_counter = ctr.recheck_total;
        fa.fallback_total = ctr.fallback_total;
        fa.fallback_reason = ctr.fallback_reason;
        fa.fb_done = nullptr;
        fa.fb_slots = 0;
        fa.rel = f32_rel_bound(x.d);
        fa.relf = static_cast<float>(2.02 * fa.rel);
        fa.ffw = static_cast<float>(2.5 * ff_rel_bound(x.d));
        I.fin_P = pi.P;
        I.fin_se = kStage;
        I.fin_pw = pi.pw;
        I.fin_wq = pi.wq;
        const bool aligned = ((reinterpret_cast<uintptr_t>(x.R) | reinterpret_cast<uintptr_t>(x.Q)) & 15) == 0;
        I.fin_nv = (aligned && (x.d & 3) == 0 && x.d <= 128) ? (x.d + 31) / 32 : 0;

        // items, and the stage each stage waits for
        auto add = [&](int stage, int64_t a0, int64_t b0) {
            by_stage[stage].push_back(BatchItem{stage, i, static_cast<int32_t>(a0), static_cast<int32_t>(b0)});
            ++I.need[stage];
        };
        for (int64_t r = 0; r < x.m; r += kPrepRows) add(kStPrepR, r, std::min<int64_t>(kPrepRows, x.m - r));
        for (int64_t r = 0; r < x.n; r += kPrepRows) add(kStPrepQ, r, std::min<int64_t>(kPrepRows, x.n - r));
        const int64_t qtiles = (x.n + 127) / 128;
        if (p.pilot) {
            for (int64_t t = 0; t < qtiles; ++t)
                for (int s = 0; s < p.S; ++s) add(kStPilot, t, s);
            for (int64_t q = 0; q < x.n; q += kThreshQueries)
                add(kStThresh, q, std::min<int64_t>(kThreshQueries, x.n - q));
        }
        for (int64_t t = 0; t < qtiles; ++t)
            for (int s = 0; s < p.S; ++s) add(kStFilter, t, s);
        const int64_t fq = 2 * static_cast<int64_t>(pi.wq);
        for (int64_t q = 0; q < x.n; q += fq) add(kStFinal, q, std::min<int64_t>(fq, x.n - q));
        add(kStFallback, 0, 0);
        I.prev[kStPrepQ] = kStPrepR;
        I.prev[kStPilot] = kStPrepQ;
        I.prev[kStThresh] = kStPilot;
        I.prev[kStFilter] = p.pilot ? kStThresh : kStPrepQ;
        I.prev[kStFinal] = kStFilter;
        I.prev[kStFallback] = kStFinal;
    }
    std::vector<BatchItem> items;
    for (int s = 0; s < kNumStages; ++s) items.insert(items.end(), by_stage[s].begin(), by_stage[s].end());
    if (items.size() > 0x7fffffffull) return cudaErrorNotSupported;

    const size_t inst_bytes = sizeof(BatchInst) * static_cast<size_t>(ninst);
    const size_t item_bytes = sizeof(BatchItem) * items.size();
    void* desc = nullptr;
    cudaError_t err = cudaMalloc(&desc, align_up(inst_bytes, 256) + item_bytes + 16);
    if (err != cudaSuccess) return err;
    err = cudaMemcpy(desc, insts.data(), inst_bytes, cudaMemcpyHostToDevice);
    if (err == cudaSuccess && item_bytes > 0)
        err = cudaMemcpy(static_cast<unsigned char*>(desc) + align_up(inst_bytes, 256), items.data(),
                         item_bytes, cudaMemcpyHostToDevice);
    if (err != cudaSuccess) {
        cudaFree(desc);
        return err;
    }
    out->desc = desc;
    out->insts = desc;
    out->items = static_cast<unsigned char*>(desc) + align_up(inst_bytes, 256);
    out->nitems = static_cast<int32_t>(items.size());
    out->ws = ws;
    out->counters_bytes = pp.counters_bytes;
    out->ready = reinterpret_cast<int32_t*>(ws + pp.off_ready);
    out->head = reinterpret_cast<int32_t*>(ws + pp.off_head);
    out->done = reinterpret_cast<int32_t*>(ws + pp.off_done);
    out->stage_ns = reinterpret_cast<unsigned long long*>(ws + pp.off_stage_ns);
    out->error_flag = ctr.error_flag;
    out->prec = prec;
    return cudaSuccess;
}

// Enqueue one run of a built batch on st: counters zeroed, the ready word set
// (unless withheld), the persistent kernel on grid_ctas CTAs.
cudaError_t persist_launch(const PersistBatch& b, int grid_ctas, bool set_ready, uint64_t wait_ns,
                           cudaStream_t st) {
    cudaError_t err = cudaMemsetAsync(b.ws, 0, b.counters_bytes, st);
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(b.ready, set_ready ? 1 : 0, sizeof(int32_t), st);
    if (err != cudaSuccess) return err;
    BatchDesc bd;
    bd.items = static_cast<const BatchItem*>(b.items);
    bd.insts = static_cast<const BatchInst*>(b.insts);
    bd.nitems = b.nitems;
    bd.head = b.head;
    bd.done = b.done;
    bd.ready = b.ready;
    bd.error_flag = b.error_flag;
    bd.wait_ns = wait_ns;
    bd.stage_ns = b.stage_ns;
    const unsigned grid = static_cast<unsigned>(std::max(1, grid_ctas));
    if (b.prec == kBF16) {
        err = allow_smem<batch_kernel<kBF16>>(kBatchDyn);
        if (err != cudaSuccess) return err;
        batch_kernel<kBF16><<<grid, kTcThreads, kBatchDyn, st>>>(bd);
    } else {
        err = allow_smem<batch_kernel<kTF32>>(kBatchDyn);
        if (err != cudaSuccess) return err;
        batch_kernel<kTF32><<<grid, kTcThreads, kBatchDyn, st>>>(bd);
    }
    return cudaGetLastError();
}

void persist_free(PersistBatch* b) {
    if (b && b->desc) cudaFree(b->desc);
    if (b) *b = PersistBatch{};
}

}  // namespace knn
