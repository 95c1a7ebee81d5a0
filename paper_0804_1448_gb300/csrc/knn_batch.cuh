// knn_batch.cuh -- host interface of the persistent batch kernel (knn_batch.cu):
// plan a batch of independent Euclidean searches in a tensor-core precision,
// build its work-item queue and instance descriptors, and enqueue it as one
// kernel launch.
#pragma once

#include <cstdint>
#include <vector>

#include "knn_internal.cuh"

namespace knn {

// One search of the batch (device pointers).  chunk > 0: split its
// references into pieces of about this many (the autotuned choice for its
// (d, k) bucket); 0: the planner's own choice.
struct PersistInst {
    const float* R;
    int64_t m;
    const float* Q;
    int64_t n;
    int32_t d, k;
    float* dist_out;
    int32_t* idx_out;
    int64_t chunk;
};

// Plans and workspace layout (byte offsets) of a batch.
struct PersistPlan {
    struct Inst {
        TcPlan plan{};
        int32_t c = 0, kp = 0, P = 0, pw = 0, wq = 0;
        size_t off_qlp = 0, off_rlp = 0, off_gmax = 0, off_lists = 0, off_counts = 0;
        size_t off_qs = 0, off_list = 0, off_scr = 0;
    };
    std::vector<Inst> inst;
    size_t off_head = 0, off_done = 0, off_rmax = 0, off_fbc = 0, off_ready = 0, off_stage_ns = 0;
    size_t counters_bytes = 0;   // [0, counters_bytes) is zeroed before every run
    size_t ws_bytes = 0;
};

// Counters of the owning handle the kernel updates.
struct PersistCounters {
    int32_t* error_flag;
    unsigned long long* recheck_total;
    unsigned long long* fallback_total;
    unsigned long long* fallback_reason;
};

// A built batch: descriptors in device memory of its own (desc), buffers in
// the workspace ws.
struct PersistBatch {
    void* desc = nullptr;
    const void* insts = nullptr;
    const void* items = nullptr;
    int32_t nitems = 0;
    unsigned char* ws = nullptr;
    size_t counters_bytes = 0;
    int32_t* ready = nullptr;
    int32_t* head = nullptr;
    int32_t* done = nullptr;
    unsigned long long* stage_ns = nullptr;   // [3][stages]: waiting ns, working ns, items (summed over CTAs)
    int32_t* error_flag = nullptr;
    int prec = 0;
};

// cudaErrorNotSupported: some instance cannot run in the persistent form
// (rows too long for the tensor-core tile, k above the fallback's limit, ...).
cudaError_t persist_plan(const std::vector<PersistInst>& in, int prec, int rerank_factor,
                         int num_sms, PersistPlan* out);
cudaError_t persist_build(const std::vector<PersistInst>& in, const PersistPlan& pp, int prec,
                          unsigned char* ws, const PersistCounters& ctr, PersistBatch* out);
cudaError_t persist_launch(const PersistBatch& b, int grid_ctas, bool set_ready, uint64_t wait_ns,
                           cudaStream_t st);
void persist_free(PersistBatch* b);
size_t persist_item_smem();
// Stages of the persistent batch: operand rows of R, of Q, pilot, threshold,
// filter, finalize, exact fallback.
constexpr int kPersistStages = 7;

}  // namespace knn
