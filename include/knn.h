/*
 * knn.h -- C ABI of the GB300 (sm_103a) brute-force k-nearest-neighbour library.
 *
 * The operation is the one of Sec. 2.1 ("Problem definition") of Garcia,
 * Debreuve and Barlaud, "Fast k Nearest Neighbor Search using GPU": given m
 * reference points R = {r_1..r_m} and n query points Q = {q_1..q_n} in R^d,
 * return for every query the k reference points nearest to it under a given
 * distance.  The brute-force method of the same section (compute all m
 * distances, sort, keep the k smallest, for every query) fixes the result;
 * this library reaches the same result without writing the n x m distance
 * matrix to memory: each distance tile is consumed on chip by a per-query
 * top-k selection.
 *
 * Conventions (the paper fixes none of them):
 *   - points are rows: R is m x d and Q is n x d, row-major, contiguous,
 *     IEEE float32;
 *   - indices are 0-based (the paper writes r_1..r_m);
 *   - every output row i holds k pairs (dist, idx) ascending by distance,
 *     equal distances ordered by the smaller index;
 *   - Euclidean results are true distances ||q - r||_2 (not squared);
 *     Manhattan results are sum_t |q_t - r_t|;
 *   - non-finite coordinates are a precondition violation: results are
 *     unspecified (they are not checked on the hot path).
 *
 * Every entry point returns a knn_status.  On any error status nothing has
 * been written to the caller's output buffers.  A handle is not thread-safe:
 * use one handle per host thread or serialise calls externally.
 */
#ifndef KNN_GB300_H
#define KNN_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct knn_ctx* knn_handle; /* opaque; owned by the library */

/*
 * Distances: the two Sec. 2.1 names ("the Euclidean or the Manhattan
 * distance"), and two more the same passage admits: the Chebyshev
 * (L-infinity) distance max_t |q_t - r_t|, and the Mahalanobis distance
 * sqrt((q - r)^T S^-1 (q - r)) for the inverse covariance S^-1 given with
 * knn_set_mahalanobis.  Manhattan and Chebyshev searches run in KNN_FP32
 * whatever the handle's precision; a Mahalanobis search is a Euclidean search
 * of whitened points (below) in the handle's precision.
 */
typedef enum { KNN_L2 = 0, KNN_L1 = 1, KNN_LINF = 2, KNN_MAHALANOBIS = 3 } knn_metric;

/*
 * Arithmetic of the distance stage.
 *   KNN_FP32: float32 on CUDA cores, distances formed from coordinate
 *             differences (sum (q-r)^2 or sum |q-r|).
 *   KNN_BF16 / KNN_TF32: Euclidean only.  The cross term q.r runs on the
 *             tensor cores (tcgen05) in bf16 or tf32 with float32
 *             accumulation, the norms are added in the epilogue
 *             (||q||^2 + ||r||^2 - 2 q.r), the best rerank_factor * k
 *             candidates per query are re-ranked with exact float32
 *             differences.  Manhattan and Chebyshev distances ignore this
 *             setting and run in KNN_FP32, and so do Euclidean searches
 *             whose rows do not fit the tensor-core tile in shared memory
 *             (d above 444 in bf16, above 220 in tf32) and searches of
 *             reference sets too small for the tensor-core pilot (m below
 *             about 2800 at k = 20, at most 4096), where the exact float32
 *             form is the faster one.
 * In every mode, candidates whose float32 distances lie within the float32
 * rounding bound of each other around the returned list are re-checked on the
 * GPU (a float-float sum, and the oracle's float64 arithmetic where that
 * cannot separate them), so ties are resolved by the exact distance.
 */
typedef enum { KNN_FP32 = 0, KNN_TF32 = 1, KNN_BF16 = 2 } knn_precision;

typedef enum {
    KNN_OK = 0,
    KNN_ERR_INVALID = 1,     /* bad argument: null pointer, k<1, k>m, d mismatch, ... */
    KNN_ERR_OOM = 2,         /* device memory could not be obtained (or is over the limit) */
    KNN_ERR_CUDA = 3,        /* a CUDA call failed; see knn_last_error() */
    KNN_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    KNN_ERR_NOREF = 5,       /* knn_search before knn_set_reference */
    KNN_ERR_BUSY = 6,        /* the handle, or its shared reference set, is in use */
    KNN_ERR_UNSUPPORTED = 7  /* valid request outside this build's limits (see KNN_K_MAX) */
} knn_status;

/* Largest k accepted by knn_search. */
#define KNN_K_MAX 1024

typedef struct {
    int32_t precision;       /* knn_precision; default KNN_FP32 */
    int32_t rerank_factor;   /* low-precision forms keep rerank_factor*k candidates; default 4 */
    int64_t workspace_limit; /* max bytes of device scratch the handle may hold; 0 = no limit */
} knn_options;

/* Fill *opt with the defaults above. */
void knn_options_default(knn_options* opt);

/*
 * Create a handle bound to CUDA device `device`.  opt may be NULL
 * (defaults).  The handle owns a CUDA stream, the device copy of the
 * reference set and a scratch workspace.
 * Errors: KNN_ERR_INVALID (out == NULL, bad option), KNN_ERR_CUDA (no such
 * device / no driver).
 */
knn_status knn_create(knn_handle* out, int device, const knn_options* opt);

/*
 * Set the reference set R (m x d, row-major float32) -- the set R of
 * Sec. 2.1.  The library COPIES R into device memory it owns (the caller
 * keeps ownership of its buffer and may free it on return) and precomputes
 * what later searches need (squared norms, the bf16/tf32 copy when the
 * handle's precision asks for one).  r_on_device = 1: R is a device
 * pointer on the handle's device; 0: a host pointer.  The call is
 * synchronous.  Replaces any previous reference set.
 * Errors: KNN_ERR_INVALID (R NULL, m < 1, d < 1), KNN_ERR_OOM, KNN_ERR_CUDA.
 */
knn_status knn_set_reference(knn_handle h, const float* R, int64_t m, int32_t d,
                             int r_on_device);

/*
 * k nearest neighbours of each of the n queries Q (n x d, row-major
 * float32) among the current reference set, under `metric` -- the search
 * of Sec. 2.1.  Writes dist_out[i*k + s] (float32) and idx_out[i*k + s]
 * (int32, 0-based), s = 0..k-1 ascending.
 *   io_on_device = 1: Q, dist_out and idx_out are device pointers valid on
 *     `cuda_stream`; the call only enqueues work and returns (asynchronous).
 *   io_on_device = 0: host pointers; the call copies Q in, searches, copies
 *     the results out and returns when they are in place (synchronous).
 *     Pinned host memory makes the copies faster; pageable works too.  In
 *     the tensor-core forms pinned Q and outputs are not copied: the kernels
 *     read Q and write the results over the CPU-GPU link in place, and from
 *     8192 queries on the search runs as two parts on two streams (the
 *     handle's second stream joins back into cuda_stream), so that the
 *     second part's queries cross the link while the first part computes.
 *     Neither changes the result.
 * cuda_stream: a cudaStream_t, or NULL for the handle's own stream.
 * n = 0 is a no-op returning KNN_OK.
 * Errors: KNN_ERR_INVALID (null pointer with n > 0, n < 0, k < 1, k > m,
 * d != the reference dimension, bad metric, KNN_MAHALANOBIS without a
 * matrix of dimension d), KNN_ERR_UNSUPPORTED (k > KNN_K_MAX), KNN_ERR_NOREF,
 * KNN_ERR_OOM, KNN_ERR_CUDA.
 */
knn_status knn_search(knn_handle h, const float* Q, int64_t n, int32_t d, int32_t k,
                      knn_metric metric, float* dist_out, int32_t* idx_out,
                      int io_on_device, void* cuda_stream);

/*
 * Wait for all work the library enqueued on this handle's device and report
 * a bounded device-side wait that gave up during it (KNN_ERR_TIMEOUT, after
 * which the flag is cleared).  The asynchronous form of knn_search reports
 * such a failure only here or in a later synchronous call.
 */
knn_status knn_sync(knn_handle h);

/*
 * Self-test of that failure detection: enqueues on the handle's stream one
 * device-side wait, bounded by limit_ms (1..1000), on a barrier nothing
 * completes -- the wait gives up, raises the handle's error flag the way a
 * search kernel does and returns -- then does knn_sync.  Returns
 * KNN_ERR_TIMEOUT when the detection works; the handle stays usable.  No
 * fault, trap or hang is involved.  Errors: KNN_ERR_INVALID, KNN_ERR_CUDA.
 */
knn_status knn_selftest_bounded_wait(knn_handle h, int32_t limit_ms);

/*
 * The plan a search would run with, without running it (host only; no GPU,
 * no handle): how knn_search of n queries against m references of dimension
 * d would be split and staged on a GPU with num_sms SMs, in the given
 * precision (knn_precision) with rerank_factor * k re-rank candidates for the
 * tensor-core forms.  For understanding performance: whether the pilot runs,
 * how many references a query tile's CTAs share, the hit-list sizes, the
 * workspace the search needs (device I/O).  KNN_MAHALANOBIS plans as the
 * Euclidean search it becomes.  Errors: KNN_ERR_INVALID (out NULL, n < 1,
 * m < 1, d < 1, k < 1, k > m, bad metric, precision or rerank_factor,
 * num_sms < 1), KNN_ERR_UNSUPPORTED (the search would be refused).
 */
typedef struct {
    int32_t tensor_cores;       /* 1: tensor-core filter (bf16/tf32); 0: float32 CUDA-core select */
    int32_t candidates;         /* candidates per query kept for the exact re-rank */
    int32_t splits;             /* reference splits (CTAs sharing one query tile) */
    int64_t chunk;              /* references per split */
    int32_t k_blocks;           /* tensor cores: 128-byte K blocks per operand row */
    int32_t stages;             /* tensor cores: depth of the reference stage ring */
    int32_t whole_tile_stages;  /* tensor cores: 1 when a stage holds a whole reference tile */
    int32_t raw_staging;        /* tensor cores: 1 float32 hit staging, 0 16-bit codes */
    int32_t pilot;              /* tensor cores: 1 pilot + threshold, 0 every reference kept */
    int32_t pilot_stride;       /* the pilot samples every stride-th reference tile */
    int32_t pilot_groups;       /* group maxima per query */
    int32_t threshold_rank;     /* which largest group maximum becomes the threshold */
    int32_t list_capacity;      /* hit-list entries per query, split and column group */
    int32_t fallback_slots;     /* scratch rows of the exact fallback */
    int64_t workspace_bytes;    /* device workspace of the search (device I/O) */
    int32_t small_select;       /* float32: 1 when each query's m distances are held in
                                   shared memory and the c nearest selected exactly (small
                                   reference sets; the tensor-core forms take this path
                                   too when their pilot would not run) */
    int32_t pilot_group_size;   /* tensor cores: references per pilot group (32; 16 or 8 when
                                   every tile is sampled and groups of 32 are too few) */
} knn_plan;

knn_status knn_explain_plan(int64_t n, int64_t m, int32_t d, int32_t k, knn_metric metric,
                            int32_t precision, int32_t rerank_factor, int32_t num_sms,
                            knn_plan* out);

/*
 * Change the handle's precision (knn_precision).  Builds the bf16/tf32
 * copy of the current reference set if one is needed.  Synchronous.
 * Errors: KNN_ERR_INVALID, KNN_ERR_OOM, KNN_ERR_CUDA.
 */
knn_status knn_set_precision(knn_handle h, int32_t precision);

/*
 * The matrix of the Mahalanobis distance (KNN_MAHALANOBIS, Sec. 2.1):
 * S_inv is a HOST pointer to a d x d symmetric positive definite matrix, the
 * inverse covariance, row-major double (the lower triangle is read).  The
 * library factors it once, S_inv = L L^T (Cholesky, in double on the host),
 * keeps L on the device in float32, and answers KNN_MAHALANOBIS searches as
 * Euclidean searches of whitened points x' = L^T x: the reference set is
 * whitened on the first such search after knn_set_reference or this call (a
 * second float32 copy, m x d, owned by this handle), the queries on every
 * search.  Each whitened coordinate is computed with a compensated dot
 * product and rounded once, so returned distances are those of the exact
 * quadratic form to within float32 rounding of the whitened coordinates.
 * S_inv = NULL forgets the matrix.  KNN_MAHALANOBIS is not available to
 * knn_search_batch, knn_search_self or knn_search_static.  Synchronous.
 * Errors: KNN_ERR_INVALID (d < 1, S_inv not positive definite or not finite),
 * KNN_ERR_UNSUPPORTED (d above 224), KNN_ERR_OOM, KNN_ERR_CUDA.
 */
knn_status knn_set_mahalanobis(knn_handle h, const double* S_inv, int32_t d);

/* Counters since knn_create (reading them synchronises the handle's work). */
typedef struct {
    int64_t searches;          /* knn_search calls that did work */
    int64_t kernel_launches;   /* this library's kernels launched */
    int64_t recheck_entries;   /* candidates re-checked in float64 */
    int64_t fallback_queries;  /* queries finished by the exact float64 pass */
    int64_t workspace_bytes;   /* device scratch currently held */
    /* why queries went to the exact float64 pass (tensor-core forms: the
       filtered list was shorter than the candidates wanted, overflowed, or
       its cut kept too many; float32 form: completeness not certified) */
    int64_t fallback_short_list;
    int64_t fallback_overflow;
    int64_t fallback_wide_cut;
    int64_t fallback_uncertified;
} knn_stats;

knn_status knn_get_stats(knn_handle h, knn_stats* out);

/*
 * Per-stage device times of the next searches.  knn_set_profiling(h, 1)
 * makes knn_search record CUDA events around each of its stages on the
 * stream it runs on; knn_get_profile() synchronises and returns, for the
 * most recent search, the milliseconds of up to `cap` stages in `ms` and
 * their names in `names` (static strings), and the number of stages in
 * *count.  Profiling adds event records only; it changes no result.
 */
knn_status knn_set_profiling(knn_handle h, int on);
knn_status knn_get_profile(knn_handle h, float* ms, const char** names, int32_t cap,
                           int32_t* count);

/*
 * Self-join with self-exclusion: for every point r_i of the current reference
 * set, its k nearest OTHER reference points (index i itself left out; other
 * points equal to r_i stay, at distance 0).  This is the neighbour relation of
 * the entropy estimate of Sec. 2.2 (rho_k(y_i) is the distance from y_i to
 * its k-th nearest neighbour among the other points).  Writes m x k outputs
 * (device pointers, knn_search's conventions and precision); asynchronous on
 * cuda_stream (NULL = the handle's stream).  Runs as a search of R against
 * itself for k + 1 neighbours and a device pass that drops each row's own
 * index (or, when more than k equal points precede it, the last entry).
 * Errors: KNN_ERR_INVALID (null pointer, k < 1, k + 1 > m, bad metric),
 * KNN_ERR_NOREF, KNN_ERR_UNSUPPORTED (k + 1 > KNN_K_MAX, KNN_MAHALANOBIS),
 * KNN_ERR_OOM, KNN_ERR_CUDA.
 */
knn_status knn_search_self(knn_handle h, int32_t k, knn_metric metric, float* dist_out,
                           int32_t* idx_out, void* cuda_stream);

/*
 * The float32 search of knn_search (returned distances from coordinate
 * differences, float64 re-check of near ties, exact fallback) for callers that cannot
 * allocate device memory when they search: frameworks that hand out every
 * device allocation from their own pool (and account for it), and
 * latency-critical paths that cannot take the device-wide synchronisation of
 * cudaMalloc/cudaFree.  The paper has no counterpart: it describes the
 * search, not its memory management.
 *
 * No handle and no allocation: R (m x d), Q (n x d), dist_out and idx_out
 * (n x k) are device pointers on the current device, valid on cuda_stream
 * (NULL = the legacy default stream); metric is KNN_L2, KNN_L1 or KNN_LINF; the results
 * follow knn_search's conventions.  The call only enqueues work
 * (asynchronous).  Intermediates live in one 32 MiB __device__ array that
 * belongs to the library's device image, so every GPU that loads the library
 * holds those 32 MiB until the process exits.
 *
 * The first call on a device looks the array's address up (once per device);
 * make that first call before any stream capture.  Every call shares the
 * array and leaves its contents there; calls that overlap on the GPU (on
 * different streams, or from different threads) race and must be serialised
 * by the caller.
 *
 * Errors: KNN_ERR_INVALID (bad argument, k > m), KNN_ERR_UNSUPPORTED when the
 * problem needs more scratch than the array holds, or k > KNN_K_MAX,
 * KNN_ERR_CUDA.  The scratch is n * S * 8 * (k + max(8, k/4)) bytes of
 * candidates, S being the number of reference splits the float32 search
 * plans for this n, m, k and the GPU's SM count (1 when the query tiles alone
 * fill the GPU, more for few queries), plus n * 4 bytes of fallback queue and
 * m * 8 bytes for the exact fallback.
 */
knn_status knn_search_static(const float* R, int64_t m, const float* Q, int64_t n, int32_t d,
                             int32_t k, knn_metric metric, float* dist_out, int32_t* idx_out,
                             void* cuda_stream);

/*
 * A second handle on the reference set of `src`, for running searches on it
 * concurrently (each handle has its own stream, workspace and counters; the
 * device copy of R, its norms and its bf16/tf32 copy are shared, read-only,
 * and live until the last handle that uses them is destroyed or given a new
 * reference set).  This is how a serving loop keeps one resident reference
 * set and overlaps requests on the GPU; the paper searches one query set at a
 * time and has no counterpart.  opt may be NULL (src's options); a non-NULL
 * opt must keep src's precision.  A shared handle cannot switch the shared
 * set to another low-precision copy (knn_set_precision then returns
 * KNN_ERR_BUSY); knn_set_reference on it detaches it from the shared set.
 * Errors: KNN_ERR_INVALID (out or src NULL, precision differs, bad option),
 * KNN_ERR_OOM, KNN_ERR_CUDA.
 */
knn_status knn_create_shared(knn_handle* out, knn_handle src, const knn_options* opt);

/*
 * Bytes of device workspace that knn_search(h, ..., n, d, k, metric, ...,
 * io_on_device, ...) needs with h's current reference set and precision
 * (written to *bytes; 0 for n = 0).  Nothing is allocated or launched.  With
 * knn_reserve, this lets a caller admit work by memory and keep allocation
 * out of the search path.
 * Errors: as knn_search's argument checks (KNN_ERR_INVALID, KNN_ERR_NOREF,
 * KNN_ERR_UNSUPPORTED); KNN_ERR_INVALID when bytes is NULL.
 */
knn_status knn_workspace_size(knn_handle h, int64_t n, int32_t d, int32_t k, knn_metric metric,
                              int io_on_device, int64_t* bytes);

/*
 * Grow h's workspace now to at least `bytes` (synchronous), so that later
 * searches needing no more than that allocate nothing.  Never shrinks it.
 * Errors: KNN_ERR_INVALID (h NULL, bytes < 0), KNN_ERR_OOM (including over
 * the handle's workspace_limit), KNN_ERR_CUDA.
 */
knn_status knn_reserve(knn_handle h, int64_t bytes);

/*
 * Batches: many independent searches (each with its own reference set)
 * handed over at once.  The paper's problem statement is one search
 * (Sec. 2.1); a batch is a list of such problems.
 */
typedef struct {
    const float* R;      /* m x d reference set (device) */
    int64_t m;
    const float* Q;      /* n x d queries (device); n = 0 is allowed */
    int64_t n;
    int32_t d;
    int32_t k;           /* 1 <= k <= m, k <= KNN_K_MAX */
    int32_t metric;      /* knn_metric */
    float* dist_out;     /* n x k (device) */
    int32_t* idx_out;    /* n x k (device) */
} knn_instance;

#define KNN_BATCH_AUTOTUNE 1  /* on a batch shape not seen before, time the launch
                                 configurations and keep the fastest (slower first call) */
#define KNN_BATCH_NO_GRAPH 2  /* enqueue the instances one after another, each planned
                                 as a lone search (the one-launch-per-instance form) */
#define KNN_BATCH_BRANCHES 4  /* a CUDA graph of the instances' own launches on parallel
                                 branches instead of the persistent kernel */

/*
 * Search every instance of inst[0..count) with the handle's precision and
 * re-rank factor (the handle's own reference set is not used), results as in
 * knn_search.  All pointers are device pointers; the call only enqueues work
 * on cuda_stream (NULL = the handle's stream) and returns (asynchronous).
 *
 * Tensor-core precisions with every instance Euclidean (the persistent form):
 * the whole batch is ONE kernel launch.  One CTA per SM stays resident and
 * pops work items -- (instance, stage, query tile or rows, reference split) --
 * from a queue in device memory: for every instance its operand copies, pilot,
 * per-query threshold, tensor-core filter, finalize and exact fallback, the
 * items of each stage after those of the stage before (a per-instance
 * counter, waited for with a bound).  The reference-split length of the
 * filter and pilot items is, per (d, k) bucket of the batch, the one
 * KNN_BATCH_AUTOTUNE found fastest for this batch shape (else the planner's
 * own choice).  The launch and its counter resets are captured in a CUDA
 * graph, cached by the batch's exact signature (shapes and pointers), so a
 * repeated batch is one cudaGraphLaunch; growing the workspace drops cached
 * graphs (they point into it).  A wait of the kernel that gives up raises the
 * handle's error flag (KNN_ERR_TIMEOUT from knn_sync).
 *
 * Otherwise (float32, another distance in the batch, or KNN_BATCH_BRANCHES):
 * the instances are planned together, given workspace slices of their own,
 * and their launches captured into one CUDA graph whose parallel branches run
 * them side by side (largest first onto the least loaded branch); the
 * configuration (branches, SMs each instance is planned to fill) is the one
 * KNN_BATCH_AUTOTUNE found for this batch shape, else a default (8 branches,
 * a quarter of the SMs each).
 * Errors: KNN_ERR_INVALID (h NULL, count < 0, inst NULL with count > 0, an
 * instance with a null pointer, m < 1, d < 1, k < 1, k > m or a bad metric),
 * KNN_ERR_UNSUPPORTED (k > KNN_K_MAX), KNN_ERR_OOM, KNN_ERR_CUDA.
 */
knn_status knn_search_batch(knn_handle h, const knn_instance* inst, int32_t count, int32_t flags,
                            void* cuda_stream);

/* How the last knn_search_batch ran. */
typedef struct {
    int32_t branches;       /* parallel graph branches (1 without a graph) */
    int32_t sm_share;       /* SMs each instance was planned to fill */
    int32_t launches;       /* kernels of the batch */
    int64_t graph_nodes;    /* nodes of its graph (0 without a graph) */
    int32_t tuned;          /* 1 if that call ran the autotuner */
    double tune_ms;         /* device time the autotuner spent */
    int32_t persistent;     /* 1: the batch ran as one persistent kernel launch */
    int32_t items;          /* persistent: work items in its queue */
} knn_batch_info;

knn_status knn_batch_info_get(knn_handle h, knn_batch_info* out);

/*
 * Where the last persistent batch run spent its time, per stage of its work
 * items -- 0 operand rows of R, 1 of Q, 2 pilot, 3 threshold, 4 filter,
 * 5 finalize, 6 exact fallback: wait_ms[s] and work_ms[s], the CTA time (summed
 * over the CTAs, from the GPU's global timer) its items spent waiting for
 * their instance's previous stage and working, and items[s], how many ran.
 * Each array holds 7 entries (HOST pointers).  Waits for the batch's stream.
 * Valid after a knn_search_batch that ran in the persistent form, until the
 * handle's next search of any kind.  The paper has no counterpart: it is the
 * measurement of this library's batching form.  Errors: KNN_ERR_INVALID,
 * KNN_ERR_UNSUPPORTED (no persistent run to report), KNN_ERR_CUDA.
 */
knn_status knn_batch_stage_times(knn_handle h, double* wait_ms, double* work_ms, int64_t* items);

/*
 * Self-test of the persistent batch kernel's bounded waits: enqueues on the
 * handle's stream one launch of the persistent kernel on a one-instance batch
 * whose "ready" word is withheld (the host never sets it), so every CTA's
 * first wait gives up after limit_ms (1..1000), raises the handle's error
 * flag and leaves without touching the batch; then does knn_sync.  Returns
 * KNN_ERR_TIMEOUT when the detection works; the handle stays usable.  No
 * fault, trap or hang is involved.  Errors: KNN_ERR_INVALID, KNN_ERR_OOM,
 * KNN_ERR_CUDA.
 */
knn_status knn_selftest_batch_queue(knn_handle h, int32_t limit_ms);

/* Release the handle and everything it owns.  NULL is accepted. */
knn_status knn_destroy(knn_handle h);

/* Static description of a status code. */
const char* knn_status_string(knn_status s);

/* Text of the last CUDA error seen by this handle ("" if none). */
const char* knn_last_error(knn_handle h);

#ifdef __cplusplus
}
#endif

#endif /* KNN_GB300_H */
