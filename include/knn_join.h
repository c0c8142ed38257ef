/*
 * knn_join.h -- C ABI of the GB300 sparse-vector KNN join library (libknnjoin.so).
 *
 * Paper: Wang, Lin, Huang, Wang, He, "Efficient K-Nearest Neighbor Join Algorithms
 * for High Dimensional Sparse Data".
 *
 * Problem (Section 3): for every vector r of R, return the k vectors s of S with the
 * largest dot(r, s) = sum_d r[d] * s[d] (eq. 1).  A sparse vector is a set of
 * features (d, w) with w > 0 in ascending d (Section 3).  This library orders equal
 * scores by ascending S id, leaves out zero scores, and pads a row that has fewer
 * than k positive scores with id -1 and score 0.
 *
 * Method: the inverted index of S (Section 4.3, Algorithm 3) split into S blocks, with
 * the threshold-based refinement of Section 4.4 (Algorithm 4): each list is ordered
 * so that the postings the refinement indexes come first, and a running k-th score
 * per query row (the row's pruneScore, which bounds MinPruneScore from below for a
 * one-row R block) picks how much of each list is scanned.  Scores of the vectors
 * found this way are completed with their unindexed features (Algorithm 4,
 * Find_Matches_IIIB) and a per-row top-k keeps the result.
 *
 * Conventions shared by every call:
 *   - Every call returns a knn_status; nothing is thrown or aborted across the ABI.
 *     On failure knn_last_error() returns a message for the calling thread.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is queued
 *     on it; calls that must read a result back on the host (sizes, validation
 *     flags) synchronise that stream, and say so.
 *   - Pointers flagged on_device are device pointers of the current CUDA device;
 *     otherwise they are host pointers (pinned or pageable).
 *   - Input arrays are owned by the caller and only read.  Output arrays are owned
 *     by the caller and must hold the stated number of elements.
 *   - Device memory the library needs for itself (an index, scratch) comes from the
 *     allocator installed with knn_set_allocator (default: cudaMallocAsync /
 *     cudaFreeAsync on the call's stream).
 */
#ifndef KNN_JOIN_H
#define KNN_JOIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KNN_OK = 0,
    KNN_EINVAL = 1,        /* an argument or an input vector breaks the rules above      */
    KNN_ENOMEM = 2,        /* the allocator returned NULL                                 */
    KNN_ECUDA = 3,         /* a CUDA runtime call failed (message in knn_last_error)      */
    KNN_ETIMEOUT = 4,      /* a bounded device-side wait gave up                          */
    KNN_EUNSUPPORTED = 5   /* valid input outside this build's limits (k, row size, ...)  */
} knn_status;

typedef enum {
    KNN_U8 = 0,   /* uint8 weights, int32 scores (exact)                                  */
    KNN_F32 = 1   /* float32 weights, float32 scores                                      */
} knn_dtype;

/* A set of sparse vectors in CSR form.
 *   indptr  int64[n_rows + 1], indptr[0] == 0, non-decreasing
 *   indices int32[indptr[n_rows]], 0 <= d < dim, strictly ascending within a row
 *   values  uint8 or float32 [indptr[n_rows]], every w > 0 (and finite)
 * Rows may be empty.  Section 3 fixes w > 0; the Section 4.4 bound needs w >= 0.   */
typedef struct {
    int64_t n_rows;
    int32_t dim;
    knn_dtype dtype;
    const int64_t* indptr;
    const int32_t* indices;
    const void* values;
    int32_t on_device;     /* 1: the three arrays are device pointers; 0: host pointers */
} knn_csr;

/* Limits of this build. */
#define KNN_MAX_K 64              /* largest k of knn_join                               */
#define KNN_MAX_LEVELS 32         /* largest number of threshold levels of an index      */
#define KNN_MAX_BLOCK 32768       /* largest S block (S vectors per block)               */

/* Allocator used for every device buffer the library owns.  `alloc` returns a device
 * pointer of at least `bytes` bytes usable on `stream`, or NULL; `release` gives it
 * back.  Passing NULL for both restores the default (cudaMallocAsync/cudaFreeAsync).
 * Process-wide; install it before building an index.                              */
typedef void* (*knn_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*knn_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);
knn_status knn_set_allocator(knn_alloc_fn alloc, knn_free_fn release, void* ctx);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* knn_last_error(void);

/* Library version string. */
const char* knn_version(void);

/* Number of CUDA kernels this library has launched in this process so far. */
int64_t knn_kernel_launch_count(void);

/* ------------------------------------------------------------------------------ */
/* Index of S (Section 4.3 inverted lists, Algorithm 3's Create_Inverted_List_IIB,  */
/* with Section 4.4's index cut precomputed for a ladder of thresholds)             */
/* ------------------------------------------------------------------------------ */

typedef struct {
    int32_t block_size;   /* S vectors per S block: power of two in [256, 32768];
                             0 = 16384 (or the next power of two >= |S| if smaller)   */
    int32_t n_levels;     /* threshold levels of the Section 4.4 cut, 1..32; 0 = 16;
                             1 = no refinement (every list scanned whole, IIB)       */
} knn_build_opts;

typedef struct knn_index knn_index;

typedef struct {
    int64_t n_rows, nnz;
    int32_t dim, block_size, n_blocks, n_levels;
    knn_dtype dtype;
    int32_t max_row_nnz;
    size_t device_bytes;  /* bytes the index holds on the device */
    size_t host_bytes;    /* bytes it holds in pinned host memory (knn_index_to_host) */
} knn_index_info;

/* Builds the index of S on the current device.
 *   S      the database vectors (host or device CSR, see knn_csr).
 *   opts   NULL for defaults.
 *   out    receives the handle; the handle owns a device copy of everything it needs
 *          (S may be freed after the call returns).
 * Dimension order for the Section 4.4 cut: descending document frequency in S, ties
 * by ascending dimension.  Synchronises `stream` (validation and sizing).
 * Errors: KNN_EINVAL for a malformed S (unsorted or repeated d, d out of range,
 * w <= 0, bad indptr), KNN_EUNSUPPORTED for more than 2^31-1 features,
 * KNN_ENOMEM, KNN_ECUDA.                                                           */
knn_status knn_join_build_index(const knn_csr* S, const knn_build_opts* opts, void* stream,
                                knn_index** out);

knn_status knn_index_get_info(const knn_index* index, knn_index_info* info);

/* Out-of-core form of Algorithm 1's block nested loop: moves every array of the index
 * into pinned, mapped host memory (on a GB300 node, the Grace CPU's memory) and frees
 * its device memory.  knn_join (and knn_join_learned) then stream the index: before
 * each S-block-synchronous launch, that launch's slice (its S blocks' bins and
 * postings, and the per-vector arrays of its S range) is copied into one of two
 * device staging buffers on a copy stream while the previous launch runs; the staging
 * memory (two slices) comes from the allocator for the duration of the call.  The
 * batched form and knn_join_noalloc read the arrays in place over the host link
 * (same results, much slower).  The build still needs device memory for the whole
 * index.  Synchronises `stream` (NULL: the build stream).  A second call does nothing.
 * Errors: KNN_ENOMEM (host allocation; the index is left unchanged), KNN_ECUDA.      */
knn_status knn_index_to_host(knn_index* index, void* stream);

/* Frees the index (device buffers go back to the allocator on its build stream, host
 * arrays are released). */
void knn_index_destroy(knn_index* index);

/* ------------------------------------------------------------------------------ */
/* Join (Algorithm 1's loop over S blocks per R row; Find_Matches of Algorithms 3/4) */
/* ------------------------------------------------------------------------------ */

typedef enum {
    KNN_MODE_IIIB = 0,    /* threshold-refined scan (Section 4.4), the default        */
    KNN_MODE_IIB = 1,     /* every list scanned whole (Section 4.3)                   */
    KNN_MODE_BF = 2       /* brute force (Algorithm 2), a baseline: every s of each S
                             block scored in full against r; same results, no posting
                             scan.  knn_join only (not the batched form).            */
} knn_mode;

typedef struct {
    knn_mode mode;
    int32_t threads;            /* threads per CTA (128..1024, multiple of 32); 0 = 512  */
    int32_t s_groups;           /* S-block groups scanned in parallel per row; 0 = auto  */
    const float* init_threshold;/* device float[n_rows] or NULL.  When given, row i keeps
                                   only vectors with score >= init_threshold[i] (a
                                   learned start for pruneScore).  NULL = 0 (strict >).  */
    int32_t* n_found;           /* device int32[n_rows] or NULL: entries returned per row
                                   (== k means the row's top-k is exact)                  */
    int64_t* postings_scanned;  /* device int64[1] or NULL: postings read, added to it   */
    int32_t outputs_on_host;    /* 1: out_ids/out_scores are host pointers; the call then
                                   synchronises `stream` before returning                */
    int32_t skip_validation;    /* 1: trust R (sorted, in range, w > 0)                   */
    float level_margin;         /* Section 4.4 cut per S block: the highest level l with
                                   M * L_l <= level_margin * theta (0 = 0.3 for a uint8
                                   index, 0.2 for float32).  Lower values scan more
                                   postings and complete fewer candidates.               */
    int64_t* stats;             /* device int64[KNN_STATS_LEN] or NULL: work counters,
                                   added to (see KNN_STAT_*)                              */
    int32_t blocks_per_launch;  /* with one group per row: S blocks per kernel launch;
                                   every launch covers all rows (0 = as many as keep one
                                   launch's postings within ~48 MB, so that they stay in
                                   L2 while every row reads them; at most 16)              */
    int32_t no_fixed_point;     /* float32 with one S-block group per row.  0 (default):
                                   each row sums its scan in int32 fixed point (scale: the
                                   largest power of two keeping |r| max|s| below 2^30); a
                                   row where one fixed-point unit exceeds 2^-23 of the
                                   smallest score it returns is joined again in fp32 by one
                                   more launch, so every returned score carries no larger
                                   an error bound than an fp32 sum (n 2^-24 relative for n
                                   terms).  1: every scan sums in fp32.                    */
} knn_join_opts;

/* Top-k of the union of several S shards (no paper counterpart: the exchange step of
 * an S-sharded join across GPUs, or of an S joined in ranges).  Part p holds, for the
 * same n_rows queries, k entries per row as knn_join returns them (ids relative to the
 * shard's first S vector, padding id -1 / score 0; device arrays); id_offset[p] (host)
 * is that shard's first S id (0..2^31-1).  Writes the k best of all parts by (score
 * desc, global id asc) with global ids, as knn_join would over the whole S; scores
 * int32 (KNN_U8) or float32 (KNN_F32).  part_ids / part_scores / id_offset are host
 * arrays of n_parts entries.  Asynchronous on `stream`.
 * Errors: KNN_EINVAL (NULL, n_parts outside [1, KNN_MAX_PARTS], k outside
 * [1, KNN_MAX_K], a bad offset).                                                      */
#define KNN_MAX_PARTS 64
knn_status knn_merge_topk(int32_t n_parts, const int32_t* const* part_ids, const void* const* part_scores,
                          const int64_t* id_offset, int64_t n_rows, int32_t k, knn_dtype dtype,
                          int32_t* out_ids, void* out_scores, void* stream);

/* Work counters of knn_join (indices into knn_join_opts.stats). */
#define KNN_STAT_BLOCK_STEPS 0      /* (row, S block) pairs processed                      */
#define KNN_STAT_CANDIDATES 1       /* accumulator entries passing the level bound          */
#define KNN_STAT_COMPLETED 2        /* entries completed over their unindexed features      */
#define KNN_STAT_PUSHED 3           /* keys pushed to the top-k merge                       */
#define KNN_STAT_MERGES 4           /* top-k merges                                         */
#define KNN_STAT_ROUNDS 5           /* extra candidate rounds (push buffer full)            */
#define KNN_STAT_RESIDUAL_FEATURES 6 /* unindexed features merged in completions            */
#define KNN_STAT_POSTINGS 7         /* postings scanned                                     */
#define KNN_STAT_SHARED_ADDS 8      /* shared-memory adds issued by the scan: every posting
                                       slot of the 16-byte chunks read, the zero-weight
                                       padding and the slots past a level's prefix included */
#define KNN_STAT_FIXED_POINT_ROWS 9 /* (row, S-block launch or group) pairs whose scan
                                       summed in fixed point (float joins; no_fixed_point)   */
#define KNN_STATS_LEN 10

/* Exact top-k of every row of R against the indexed S.
 *   index       built by knn_join_build_index (same dim and dtype as R).
 *   R           query vectors (host or device CSR).
 *   k           1..KNN_MAX_K.
 *   out_ids     int32[n_rows * k]: S ids, row-major, best first, -1 padding.
 *   out_scores  int32 (KNN_U8) or float (KNN_F32) [n_rows * k], 0 padding.
 * Row i lists min(k, #{s : dot(r_i, s) > 0}) entries (with init_threshold: those with
 * dot >= init_threshold[i]) ordered by (score desc, id asc).
 * Synchronises `stream` (it reads R's size and longest row back to size the launch;
 * when R's longest rows need a shared-memory layout above 110 KB, i.e. one CTA per SM,
 * it also reads back how many rows fit a smaller one: those rows then run in launches
 * of their own at two CTAs per SM, the long rows in launches with the full layout).
 * Errors: KNN_EINVAL (bad R, dim/dtype mismatch, k < 1), KNN_EUNSUPPORTED (k > 64,
 * a row too long for one CTA's shared memory, u8 scores that could overflow int32),
 * KNN_ENOMEM, KNN_ECUDA.                                                           */
knn_status knn_join(const knn_index* index, const knn_csr* R, int32_t k,
                    const knn_join_opts* opts, int32_t* out_ids, void* out_scores,
                    void* stream);

/* ------------------------------------------------------------------------------ */
/* Batched joins (no paper counterpart: many independent joins of Section 3 in one   */
/* persistent launch, replayed as a CUDA graph)                                     */
/* ------------------------------------------------------------------------------ */

typedef struct {
    const knn_index* index;   /* this join's S                                        */
    knn_csr R;                /* its queries, in device memory (on_device = 1)        */
    int32_t k;                /* 1..KNN_MAX_K                                         */
    int32_t* out_ids;         /* device int32 [R.n_rows * k]                          */
    void* out_scores;         /* device int32 / float [R.n_rows * k]                  */
} knn_job;

typedef struct {
    knn_mode mode;
    int32_t threads;            /* threads per CTA for every job, power of two; 0 = 512.
                                   Every job's S block must lie in [4*threads, 64*threads]. */
    int32_t blocks_per_group;   /* S blocks per work item; 0 = as blocks_per_launch's default,
                                   per job (~48 MB of postings, at most 16)                */
    float level_margin;         /* as in knn_join_opts (0 = 0.3, 0.2 for a float32 index)  */
    int32_t use_graph;          /* knn_batch_create: capture the launch into a CUDA graph   */
    int32_t skip_validation;    /* 1: trust every R                                          */
    int64_t* stats;             /* device int64[KNN_STATS_LEN] or NULL (all jobs together)   */
    int64_t wait_spins;         /* bound of a work item's wait for its row's previous group,
                                   in ~128 ns sleeps (0 = 2^24); past it the item gives up and
                                   knn_batch_check reports KNN_ETIMEOUT                        */
    int32_t test_never_publish; /* test hook: groups never announce completion, so every wait
                                   runs out (exercises the timeout path without a fault)      */
} knn_batch_opts;

typedef struct knn_batch knn_batch;   /* a prepared batch (validated jobs, work items, scratch) */

typedef struct {
    int64_t work_items;       /* (job, S-block group, row) items of one run              */
    int32_t ctas, threads;    /* persistent grid (the largest of its launches)            */
    int64_t shared_bytes;     /* dynamic shared memory per CTA (the largest)              */
    int32_t graph;            /* 1 if runs replay a captured CUDA graph                  */
    int32_t kernels_per_launch;
} knn_batch_info;

/* Prepares n_jobs joins: validates each R (synchronises `stream`), splits each job's S
 * blocks into groups of blocks_per_group, orders the work items (largest first) and,
 * with use_graph, captures the launch sequence into a CUDA graph.  The jobs' arrays
 * must stay valid and unchanged in size while the batch exists; R's column indices and
 * values may change between launches, its row lengths (indptr) may not: a row longer
 * than at creation is not joined, and knn_batch_check reports KNN_EINVAL.  A job whose
 * longest rows need a shared-memory layout above 110 KB (one CTA per SM) is split once
 * here (one read-back): its rows that fit a layout within 110 KB run in a persistent
 * launch with the other such jobs at two CTAs per SM, the longer rows in a launch of
 * their own.  Float batches run two persistent passes per launch: every row in fixed
 * point (as knn_join_opts.no_fixed_point = 0 describes), then the rows it flagged in
 * fp32.                                                                              */
knn_status knn_batch_create(int32_t n_jobs, const knn_job* jobs, const knn_batch_opts* opts,
                            void* stream, knn_batch** out);
/* Runs every job (asynchronously on `stream`): one persistent kernel per launch class
 * takes the work items from a counter, in order, round by round (S-block group g of
 * every job, then group g+1); a row's group g starts from the top-k its group g-1 left
 * (a bounded wait if that item is still running).  Results land in each job's outputs
 * exactly as knn_join would write them.                                             */
knn_status knn_batch_launch(knn_batch* batch, void* stream);
/* Synchronises `stream` and reports the last run: KNN_EINVAL if a row had more
 * features than when the batch was made, KNN_ETIMEOUT if a work item gave up its
 * bounded wait for the previous S-block group of its row (that row's outputs are then
 * incomplete), else KNN_OK.                                                         */
knn_status knn_batch_check(const knn_batch* batch, void* stream);
knn_status knn_batch_get_info(const knn_batch* batch, knn_batch_info* info);
void knn_batch_destroy(knn_batch* batch);
/* create (without a graph) + launch + synchronise + destroy                         */
knn_status knn_join_batched(int32_t n_jobs, const knn_job* jobs, const knn_batch_opts* opts,
                            void* stream);

/* ------------------------------------------------------------------------------ */
/* Learned start threshold (not in the paper: it generalises Section 4.4's           */
/* MinPruneScore, a threshold derived from earlier work, to one predicted per query) */
/* ------------------------------------------------------------------------------ */

typedef struct knn_model knn_model;   /* opaque; owns its device parameters */

typedef struct {
    uint64_t seed;        /* initial weights and the sketch's hash seed */
} knn_model_opts;

typedef struct {
    int32_t epochs;       /* 0 = 20 */
    int32_t batch;        /* rows per step; 0 = 512 */
    float lr;             /* Adam step size; 0 = 1e-3 */
    float quantile;       /* pinball-loss quantile q in (0,1); 0 = 0.1.  Low q makes the
                             prediction sit below the true k-th score more often.     */
    uint64_t seed;        /* batch order */
} knn_train_opts;

/* Creates a model: sketch of 516 values per query (512 signed hash buckets of the
 * features, normalised by ||r||_2, and log1p of nnz, weight sum, ||r||_2, max weight)
 * -> 256 -> 256 -> 1 with ReLU, BF16 weights, FP32 accumulation.  It predicts
 * log(k-th best score).                                                            */
knn_status knn_threshold_model_create(const knn_model_opts* opts, void* stream, knn_model** out);
void knn_threshold_model_destroy(knn_model* model);

/* Trains on queries Q (host or device CSR) and their exact k-th best scores
 * (device float[Q.n_rows], from knn_join; rows with no k-th score, value 0, are
 * skipped) with the pinball loss at the given quantile and Adam, on the GPU.
 * final_loss (host, may be NULL) receives the last epoch's mean loss.  Synchronises. */
knn_status knn_threshold_model_train(knn_model* model, const knn_csr* Q, const float* kth_scores,
                                     const knn_train_opts* opts, float* final_loss, void* stream);

/* out_tau: device float[R.n_rows], the predicted k-th best score of each row. */
knn_status knn_threshold_model_predict(const knn_model* model, const knn_csr* R, float* out_tau,
                                       void* stream);

/* Calibrates the multiplier applied to the predictions: on held-out queries Q with
 * their exact k-th best scores (device float[Q.n_rows], 0 = no k-th score), picks the
 * largest tau_scale such that at most a fraction miss_rate of Q would start above its
 * k-th score (those rows need knn_join_learned's fallback; rows without a k-th score
 * always do).  The value (rank floor(miss_rate * n) of kth / prediction, less a
 * relative 1e-6 so that rounding cannot lift a row at that rank over) is kept in
 * the model, saved with its parameters, used by knn_join_learned when its tau_scale
 * is 0, and written to *out_scale (host, may be NULL).  Synchronises `stream`.      */
knn_status knn_threshold_model_calibrate(knn_model* model, const knn_csr* Q, const float* kth_scores,
                                         float miss_rate, float* out_scale, void* stream);

/* Save / load: all parameters, optimiser state and the calibrated multiplier as one
 * host buffer.  With host_buf = NULL, get_params only reports the size in *needed.  */
knn_status knn_threshold_model_get_params(const knn_model* model, void* host_buf, size_t bytes,
                                          size_t* needed);
knn_status knn_threshold_model_set_params(knn_model* model, const void* host_buf, size_t bytes);

typedef struct {
    knn_join_opts join;   /* options of both passes (init_threshold, n_found are set here) */
    float tau_scale;      /* multiplies the predictions (0 = the model's calibrated
                             multiplier, 1 if it was never calibrated)                  */
    const float* tau;     /* device float[n_rows]: start thresholds to use instead of the
                             model's (the model may then be NULL)                       */
} knn_learned_opts;

typedef struct {
    int64_t rows;           /* rows joined                                              */
    int64_t fallback_rows;  /* rows rejoined with the plain threshold (found < k)       */
} knn_learned_stats;

/* Exact top-k like knn_join, starting each row from a predicted threshold: every s with
 * score >= tau is kept; a row that ends with k entries is exact, the others are joined
 * again with the plain threshold on the device.  Same outputs and errors as knn_join;
 * stats (host, may be NULL).  Synchronises `stream`.                                */
knn_status knn_join_learned(const knn_index* index, const knn_model* model, const knn_csr* R,
                            int32_t k, const knn_learned_opts* opts, int32_t* out_ids,
                            void* out_scores, knn_learned_stats* stats, void* stream);

/* Test and inspection hooks of the model's kernels (no paper counterpart).
 *   knn_gemm_bf16: C[m*scm + n*scn] (+)= sum_k A[m*sam + k*sak] * B[k*sbk + n*sbn] on
 *     the tcgen05 tensor cores (bf16 inputs, fp32 accumulation in tensor memory), all
 *     device pointers; synchronises `stream`; KNN_ETIMEOUT if a bounded wait for the
 *     tensor core gave up (the model calls report the same).
 *   knn_threshold_sketch: device bf16 [R.n_rows][528] sketches (columns 516.. are 0).
 *   knn_threshold_model_forward_backward: one forward and backward pass on device bf16
 *     inputs x [B][528] and targets (log k-th scores) at a quantile; writes device
 *     predictions [B] and gradients of the mean loss [n_params].
 *   knn_threshold_model_params: device pointer to the fp32 parameters
 *     (W1 [256][528], b1 [256], W2 [256][256], b2 [256], w3 [256], b3 [1]).       */
knn_status knn_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, int64_t sam, int64_t sak,
                         const void* B, int64_t sbk, int64_t sbn, float* C, int64_t scm, int64_t scn,
                         int32_t accumulate, void* stream);
knn_status knn_threshold_sketch(const knn_model* model, const knn_csr* R, void* out_x_bf16,
                                void* stream);
knn_status knn_threshold_model_forward_backward(knn_model* model, const void* x_bf16,
                                                const float* target, int64_t B, float quantile,
                                                float* out_pred, float* out_grads, void* stream);
knn_status knn_threshold_model_params(const knn_model* model, const float** params, int64_t* n);

/* ------------------------------------------------------------------------------ */
/* Allocation-free join.  The paper has no counterpart: this is an engineering      */
/* variant of knn_join for callers that cannot let a library allocate device memory */
/* during a call -- e.g. a server that has split the GPU between its own fixed      */
/* pools, or a latency-critical loop that must not pay for an allocation or for the */
/* device-wide synchronisation a free can cause.                                    */
/* ------------------------------------------------------------------------------ */

/* Size of the one scratch array (a file-scope __device__ array) the call works in.
 * Every GPU that loads the library holds it until the process exits.               */
#define KNN_NOALLOC_SCRATCH_BYTES (16u << 20)

/* Same result, arguments and errors as knn_join, with these differences:
 *   - allocates nothing: no cudaMalloc/cudaFree and no allocator-hook call; the
 *     scratch (a check record of R and the top-k keys each row carries between
 *     S-block launches) is the library's fixed array;
 *   - R must be in device memory, outputs are device memory (outputs_on_host = 0);
 *   - rows are always scanned with one S-block group per row (s_groups is ignored);
 *   - float scans always sum in fp32 (no_fixed_point is taken as 1: the fixed-point path
 *     needs a per-row flag array), so float scores may differ from knn_join's in the
 *     last bits;
 *   - n_rows * k must not exceed (KNN_NOALLOC_SCRATCH_BYTES - 256) / 8 = 2,097,120,
 *     else KNN_EUNSUPPORTED with a message naming the limit.
 * Set-up: the first call on a device (with that device current) looks up the array's
 * device address with cudaGetSymbolAddress and keeps it.  Every call, the first and
 * the later ones, synchronises `stream`: it reads R's size and longest row back to the
 * host.
 * All calls share the array and it keeps the last call's contents: calls that overlap
 * on the GPU (other streams or host threads) race on it and must be serialised by the
 * caller.                                                                           */
knn_status knn_join_noalloc(const knn_index* index, const knn_csr* R, int32_t k,
                            const knn_join_opts* opts, int32_t* out_ids, void* out_scores,
                            void* stream);

/* ------------------------------------------------------------------------------ */
/* MS/MS spectra as sparse vectors (Section 5's preprocessing; host code, no GPU)    */
/* ------------------------------------------------------------------------------ */
/* Section 5 makes each spectrum one sparse vector: each peak is a feature, its m/z
 * times 10 is the dimension index and its intensity the value.  These calls read peak
 * lists in the MGF or MS2 text formats and build that CSR on the host, ready for
 * knn_join_build_index (S) or knn_join (R).
 *   MGF: spectra between "BEGIN IONS" and "END IONS"; KEY=VALUE header lines inside
 *        (TITLE, PEPMASS, CHARGE, ...) and peak lines "m/z intensity [charge]".
 *   MS2: "H" header lines, then per spectrum an "S" line, "I"/"Z"/"D" lines and peak
 *        lines "m/z intensity".
 * LF or CRLF line ends, space- or tab-separated fields, blank lines and lines starting
 * with '#', ';' or '!' ignored; numbers as strtod reads them (C locale).  Row i is the
 * i-th spectrum of the input; a spectrum without kept peaks is an empty row.
 * Choices the paper leaves open (each settable below):
 *   - dimension = floor(m/z * mz_scale); a product within 2^-20 below an integer counts
 *     as that integer (so decimal m/z such as 0.7 lands in the bin its digits name);
 *   - peaks of one spectrum in the same dimension: the largest intensity, or the sum
 *     (in file order);
 *   - peaks with intensity <= min_intensity are dropped (weights must be > 0);
 *   - weights: the intensity as float32, or uint8 ceil(100 * I / I_max) with I_max the
 *     spectrum's largest merged intensity (1..100).                                   */
typedef enum {
    KNN_SPECTRA_AUTO = 0,   /* MGF if the first line is BEGIN IONS or KEY=VALUE, MS2 if H/S */
    KNN_SPECTRA_MGF = 1,
    KNN_SPECTRA_MS2 = 2
} knn_spectra_format;

typedef enum { KNN_MERGE_MAX = 0, KNN_MERGE_SUM = 1 } knn_spectra_merge;
typedef enum { KNN_SPECTRA_F32 = 0, KNN_SPECTRA_U8 = 1 } knn_spectra_weights;

typedef struct {
    knn_spectra_format format;
    double mz_scale;              /* > 0; 0 = 10 (Section 5)                                  */
    knn_spectra_merge merge;      /* 0 = largest intensity                                    */
    knn_spectra_weights weights;  /* 0 = float32 intensities                                  */
    int32_t dim;                  /* > 0: the vectors' dimension, a peak at or past it is an
                                     error (give R and S the same dim); 0 = 1 + the largest
                                     dimension found                                          */
    double min_intensity;         /* >= 0; peaks with intensity <= it are dropped (0 = keep
                                     every positive peak)                                     */
    int64_t chunk_bytes;          /* >= 0; inputs are cut at spectrum starts into chunks of
                                     about this many bytes that host threads parse side by
                                     side (0 = 4 MB); the result does not depend on it        */
} knn_spectra_opts;

typedef struct {
    int64_t n_spectra;   /* rows                                                               */
    int64_t n_peaks;     /* peak lines read                                                    */
    int64_t n_features;  /* features kept (nnz)                                                */
    int64_t n_dropped;   /* peaks dropped: intensity <= min_intensity (or below float32's
                            smallest positive value)                                          */
    int64_t n_merged;    /* peaks merged into another peak's dimension                         */
    int32_t dim;
    knn_dtype dtype;
} knn_spectra_info;

typedef struct knn_spectra knn_spectra;   /* parsed spectra: a host CSR the handle owns  */

/* Parses `len` bytes of MGF or MS2 text.
 * Errors: KNN_EINVAL (malformed input: the message names the line; a negative or
 * non-finite m/z, a non-finite intensity, a dimension at or past opts->dim, a bad
 * option), KNN_EUNSUPPORTED (a dimension past int32, an intensity past float32),
 * KNN_ENOMEM (host allocation).  On error *out is NULL.                              */
knn_status knn_spectra_parse(const char* text, size_t len, const knn_spectra_opts* opts,
                             knn_spectra** out);
/* Reads the file at `path` and parses it as knn_spectra_parse does (KNN_EINVAL if it
 * cannot be opened or read).                                                         */
knn_status knn_spectra_read(const char* path, const knn_spectra_opts* opts, knn_spectra** out);
/* The spectra as a host CSR (on_device = 0): the arrays belong to `sp` and stay valid
 * until knn_spectra_free.  dtype KNN_F32 or KNN_U8 as opts->weights asked.            */
knn_status knn_spectra_csr(const knn_spectra* sp, knn_csr* out);
knn_status knn_spectra_get_info(const knn_spectra* sp, knn_spectra_info* info);
void knn_spectra_free(knn_spectra* sp);

#ifdef __cplusplus
}
#endif

#endif /* KNN_JOIN_H */
