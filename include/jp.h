/*
 * jp.h -- C-ABI of the GB300 join-project library (libjp.so).
 *
 * The library evaluates, on one GPU, the two join-project queries of
 * "Fast Join Project Query Evaluation using Matrix Multiplication"
 * (Deep, Hu, Koutris):
 *
 *   two-path (Section 2.1)   Q(x,z)         = R(x,y), S(z,y)
 *   star     (Section 2.1)   Q*_k(x1..xk)   = R1(x1,y), ..., Rk(xk,y)
 *
 * with set semantics (SELECT DISTINCT, Example 1).  Both follow the
 * heavy/light split of Algorithm 1 (Section 3.1) and of the star algorithm
 * (Section 3.2): tuples with a light value are joined by a worst-case optimal
 * expansion over CSR neighbour lists and deduplicated per x; tuples whose
 * values are all heavy become 0/1 matrices whose product (Section 2.2,
 * "Join-Project as Matrix Multiplication") runs on the tensor cores; the two
 * parts are united per output row.  The result is exact: every distinct
 * tuple, sorted lexicographically as signed int32, with no approximation.
 *
 * Conventions shared by every entry point:
 *  - All pointers in jp_rel are DEVICE pointers, or HOST pointers (pageable
 *    or pinned), detected per call; host inputs are copied to the device
 *    inside the call.  Inputs are borrowed for the duration of the call and
 *    never written.  Columns are SoA int32 arrays of n entries; any int32
 *    value is allowed (negatives included); duplicate tuples are allowed and
 *    removed (relations are sets).
 *  - Work is issued on the context's stream.  The calls return after the
 *    result count is known; result columns are then ready on that stream.
 *  - Every call returns JP_OK (0) or a negative JP_E* code and never aborts,
 *    traps or prints.  jp_last_error() gives a one-line message.  There is
 *    no CPU fallback: without a usable GPU the calls fail with JP_ECUDA.
 *  - Device memory comes from the jp_alloc_fn/jp_free_fn pair given to
 *    jp_create (the Python binding passes PyTorch's caching allocator); with
 *    NULL the library uses stream-ordered cudaMallocAsync/cudaFreeAsync.
 *    The context keeps a workspace between calls and grows it on demand.
 */
#ifndef JP_H
#define JP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define JP_OK            0
#define JP_EINVAL       -1   /* bad argument (NULL pointer, n < 0, k out of range, ...) */
#define JP_ENOMEM       -2   /* the allocator returned NULL */
#define JP_ECUDA        -3   /* a CUDA call failed (message in jp_last_error) */
#define JP_EOVERFLOW    -4   /* a device-side capacity check failed; nothing was written out of bounds */
#define JP_ETIMEOUT     -5   /* a bounded device-side wait ran out; the kernel stopped and returned */
#define JP_EUNSUPPORTED -6   /* the device is not an sm_103 GPU, or a size exceeds a stated limit */

/* Threshold modes for jp_set_threshold (Section 3.1, Section 5). */
#define JP_FIXED        0    /* use the given Delta1, Delta2 (clamped to [1, N]) */
#define JP_CLOSED_FORM  1    /* Lemma 3's minimiser of the omega = 2 cost, with the Section 5 output estimate */
#define JP_COST_MODEL   2    /* Algorithm 3 (Section 5) with GPU-calibrated constants */
#define JP_LEARNED      3    /* thresholds predicted by the model set with jp_set_predictor,
                                kept unless the cost model (Algorithm 3's) prices them above
                                3 x its own choice, which is then used instead */

typedef struct jp_ctx jp_ctx;

/* One binary relation R(x, y) as two int32 columns of n entries. */
typedef struct {
    const int32_t* x;   /* first attribute (x, z or x_i) */
    const int32_t* y;   /* join attribute y */
    int64_t n;          /* number of tuples (duplicates allowed), >= 0 */
} jp_rel;

/* Query result.  col[i] holds attribute i of every output tuple (two-path:
 * col[0] = x, col[1] = z; star: col[i] = x_{i+1}); count tuples, sorted
 * lexicographically as signed int32.  Columns are device memory owned by the
 * library until jp_result_free; they live in one allocation. */
typedef struct {
    int32_t* col[8];
    int64_t count;
    int32_t k;          /* number of columns */
    void* _block;       /* library-owned allocation backing the columns */
    size_t _bytes;
} jp_result;

/* Per-call statistics of the last query (jp_get_stats). */
typedef struct {
    int64_t n_r, n_s;          /* distinct tuples of R and S after normalisation */
    int64_t dom_x, dom_y, dom_z;
    double  out_join;          /* |OUT_join| = sum_y deg_R(y) deg_S(y) (Section 5) */
    double  out_estimate;      /* Section 5 estimate of |OUT| */
    int64_t delta1, delta2;    /* thresholds used */
    int32_t threshold_mode;
    int64_t u, v, w;           /* heavy x, heavy y, heavy z counts (matrix dims) */
    int64_t light_candidates;  /* light join size enumerated before dedup */
    int64_t out_count;         /* |OUT| */
    int64_t heavy_pairs;       /* nonzeros of the heavy product (0 if not counted) */
    int64_t kernel_launches;   /* kernels the library launched for the query */
    int64_t light_x[8];        /* x values per light class: 0 warp sort (c <= 256), 1 bucket sort
                                  (c <= 2048), 2 single list copied in place, 3 bitmap (larger c,
                                  and every heavy x), 4 and 5 merge of sorted lists (c <= 4096,
                                  c <= 8192), 6 bitmap hubs (>= 128 lists or >= 65536
                                  candidates), 7 merge of sorted lists (c <= 2048); the bucket
                                  sort (1) keeps rows of c <= 2048 with more than 64 lists */
    int64_t light_cand[8];     /* candidates enumerated per light class */
    int64_t light_deg[8];      /* neighbour-list entries read per light class */
    double  ms_total;          /* host wall time of the call */
    double  ms_pass[16];       /* device ms (CUDA events on the query stream) of:
                                  0 index build, 1 threshold selection, 2 partition,
                                  3 matrix build, 4 heavy GEMM kernel, 5 light
                                  classification, 6-9 light kernels (warp sort,
                                  bucket sort, merge, bitmap+union), 10 output count,
                                  11 output placement kernel, 12 whole query; for
                                  jp_two_path_counts 4 is the counting product, and 13
                                  candidate fill, 14 sort and run lengths, 15 heavy rows,
                                  merge and output, each summed over the x ranges */
    int64_t learned_judged;    /* JP_LEARNED only: 1 the model's thresholds were used, 2 the cost
                                  model judged them too costly (modelled cost above judge x that
                                  of Algorithm 3's thresholds, or a heavy block -- FP8 operands
                                  and the product's bit matrix -- above half of the free device
                                  memory) and Algorithm 3's were used; else 0 */
    int64_t filter_pairs;      /* jp_two_path_filter only: distinct candidate pairs of T */
    int64_t filter_query_out;  /* jp_two_path_filter only: |OUT| of the query on the reduced R and S
                                  (out_count is then the number of pairs of T answered) */
    int64_t count_ranges;      /* jp_two_path_counts only: ranges of x whose light candidates were
                                  sorted in one pass each (ms_pass[13..15] sum their phases) */
    int64_t count_light_pairs; /* jp_two_path_counts only: distinct (x, z) among the light candidates
                                  (heavy_pairs: nonzero entries of the heavy product) */
    int64_t gemm_tile;         /* tile width of the heavy product (128 or 256; 0: no product) */
} jp_stats;

typedef void* (*jp_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void  (*jp_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

/* Create a context on `device`, issuing work on `stream` (a cudaStream_t, NULL
 * = legacy default stream).  alloc/free may both be NULL (see above).
 * Fails with JP_EUNSUPPORTED when the device is not compute capability 10.3. */
int jp_create(jp_ctx** ctx, int device, void* stream, jp_alloc_fn alloc, jp_free_fn release,
              void* user);

/* Release the context's workspace and the context itself (NULL is a no-op). */
void jp_destroy(jp_ctx* ctx);

/* Choose how Delta1 (y threshold) and Delta2 (x/z threshold) are picked
 * (Section 3.1: a tuple is light when a value's degree is <= its threshold).
 * delta1/delta2 are used in JP_FIXED mode only and must be >= 1. */
int jp_set_threshold(jp_ctx* ctx, int mode, int64_t delta1, int64_t delta2);

/* Constants of the cost-based optimizer (Section 5, Table 2, Algorithm 3), used by
 * JP_COST_MODEL and by the judge of JP_LEARNED.  Algorithm 3 starts at Delta1 = N,
 * Delta2 = max(N Delta1 / OUT_est, 1) and multiplies Delta1 by (1 - eps) while the modelled cost
 *   T_I sum(y_D1) + T_I sum(x_D2) + T_m |dom x| + T_s cdfx(y_D1) |dom x|
 *   + [u, v, w > 0] (2 u v w / mm_rate + mm_fixed + T_m (u v + u w))
 * does not grow, and returns the last thresholds before it grew (floored, clamped to [1, N]);
 * u, v, w are the heavy x, y and z counts at those thresholds, the sums are over light y
 * (max(deg_R, deg_S) <= Delta1: deg_R deg_S, and deg_R for cdfx) and light x (deg <= Delta2:
 * sum over the x's y of deg_S).  N is max(|R|, |S|) after R's tuples with no y in S are
 * dropped.  When OUT_join <= wcoj_factor N every value is light (Delta1 = Delta2 = N).
 * Times are in seconds; only their ratios matter. */
typedef struct {
    double T_I;          /* per light candidate inserted into a deduplication structure, >= 0 */
    double T_m;          /* per matrix element / per-x structure set up, >= 0 */
    double T_s;          /* per sequential step of a scan of the light-y list, >= 0 */
    double mm_rate;      /* heavy product: 2 u v w operations at this rate (per second), > 0 */
    double mm_fixed;     /* heavy product: fixed time, >= 0 */
    double eps;          /* descent step, 0 < eps < 1 */
    double wcoj_factor;  /* plain worst-case optimal join when OUT_join <= wcoj_factor N, >= 0 */
    double judge;        /* JP_LEARNED keeps the model's thresholds unless they cost more than
                            judge times Algorithm 3's choice (or their heavy block does not
                            fit in half of the free device memory), >= 1 */
} jp_cost_model;

/* Replace the context's constants (copied; NULL restores the defaults: T_I = 0,
 * T_m = 1.34e-12, T_s = 5.04e-16, mm_rate = 3.85e15, mm_fixed = 1.46e-4, eps = 0.05,
 * wcoj_factor = 20, judge = 3; the first five fitted by least squares to whole-query times
 * measured on GB300 over a 7 x 7 grid of fixed thresholds on 789 power-law self-joins of 1e5 to
 * 5e6 tuples).  A value out of range gives JP_EINVAL and keeps the old ones. */
int jp_set_cost_model(jp_ctx* ctx, const jp_cost_model* model);
/* The context's current constants. */
int jp_get_cost_model(const jp_ctx* ctx, jp_cost_model* model);

/* Tile of the heavy product (the tcgen05 kernel computes one tile of 128 heavy x by `width`
 * heavy z per CTA): width 128 or 256, or 0 (auto, the default): 128 when the product has at
 * most auto_max_tiles tiles of 128 x 256 (small products then spread over more SMs), else 256.
 * The default crossover comes from the tile autotuner (paper_2002_12459_gb300/tune.py), which
 * times both widths on products of many shapes.  JP_EINVAL for another width or a negative
 * count.  jp_two_path_counts always uses width 256. */
int jp_set_gemm_tile(jp_ctx* ctx, int width, int64_t auto_max_tiles);
int jp_get_gemm_tile(const jp_ctx* ctx, int* width, int64_t* auto_max_tiles);

/* Change the stream of subsequent calls. */
int jp_set_stream(jp_ctx* ctx, void* stream);

/* Two-path query Q(x,z) = R(x,y), S(z,y) (Section 2.1, Algorithm 1).
 * S == NULL means S = R (self-join).  On success *out holds count sorted
 * distinct (x, z) pairs, k = 2.  R->n + S->n must stay below 2^31. */
int jp_two_path(jp_ctx* ctx, const jp_rel* R, const jp_rel* S, jp_result* out);

/* The two-path query of jp_two_path written into caller-owned columns: out_x and out_z hold
 * cap entries each and may be device memory of the context's device or host memory the GPU
 * can write (pinned with cudaHostAlloc or cudaHostRegister, or any host memory on a system
 * whose GPU accesses pageable memory).  The output kernel writes host columns directly over
 * the host link: no device copy of the result is made.  *count (host) receives |OUT|; when it
 * exceeds cap nothing is written, JP_EOVERFLOW is returned and *count keeps |OUT| so the
 * caller can retry with larger buffers (any other failure leaves *count = 0).  Inputs,
 * thresholds and errors as jp_two_path; JP_EINVAL when a buffer is not writable by the GPU.
 * The call returns when the columns are written. */
int jp_two_path_into(jp_ctx* ctx, const jp_rel* R, const jp_rel* S, int32_t* out_x, int32_t* out_z,
                     int64_t cap, int64_t* count);

/* Measured dense tensor rates of this GPU, the denominators of the heavy product's roofline:
 * *fp8_tflops from tcgen05 kind::f8f6f4 MMAs of the product's 128x256x32 shape on operands in
 * shared memory (one CTA per SM, no loads), *int8_mma_sync_tflops from the legacy
 * mma.sync m16n8k32 s8 path.  Takes about 50 ms. */
int jp_measure_peaks(jp_ctx* ctx, double* fp8_tflops, double* int8_mma_sync_tflops);

/* Self-test of failure detection: a kernel waits, with the bounded wait every device-side
 * wait of the library uses (the heavy product's mbarrier waits), on an mbarrier that nothing
 * arrives at.  The wait runs out after wait_ns (1 .. 5e9), the kernel records the timeout in
 * the context's status word and returns, and the call returns JP_ETIMEOUT; the context stays
 * usable.  Any other return code means the mechanism failed. */
int jp_selftest_wait(jp_ctx* ctx, int64_t wait_ns);

/* Batch of two-path self-joins Q_q(x,z) = R_q(x,y), R_q(z,y), q = 0..nq-1, evaluated in
 * one pass of the pipeline (each pass one launch over all queries).  Every value is tagged
 * with its query ((query, value) pairs are dictionary-encoded), so the batch is the single
 * self-join of the disjoint union: no pair mixes two queries, and the thresholds are chosen
 * for the union by the context's mode.
 *   all      the queries' tuples one after another (device or host columns, as jp_two_path);
 *   qoff     host, nq + 1 entries: query q holds tuples [qoff[q], qoff[q+1]); qoff[0] = 0,
 *            qoff[nq] = all->n, non-decreasing (empty queries are allowed);
 *   out      one result (k = 2) holding the queries' sorted distinct pairs, query after query;
 *   out_off  host, nq + 1 entries, receives where each query's pairs start (out_off[nq] =
 *            out->count).
 * Errors as jp_two_path; JP_EINVAL for bad offsets. */
int jp_two_path_batch(jp_ctx* ctx, const jp_rel* all, int32_t nq, const int64_t* qoff,
                      jp_result* out, int64_t* out_off);

/* Boolean set intersection queries in one batch (Section 3.3): every candidate pair (a, b) of
 * T asks whether R(a, .) and S(b, .) share a y; the batch is the query
 * Q_batch(x,z) = R(x,y), S(z,y), T(x,z).  As in the paper's experiments, R is reduced to the
 * tuples whose x occurs in T and S to those whose z occurs in T, the two-path query runs on the
 * reduced relations (Algorithm 1, the context's threshold mode), and its output is intersected
 * with T.
 *   T      the candidate pairs: T->x holds the a (x) values, T->y the b (z) values; device or
 *          host columns as R; duplicates allowed; T->n < 2^31;
 *   S      NULL means S = R;
 *   out    the sorted distinct pairs of T whose sets intersect (k = 2).
 * Errors as jp_two_path; JP_EINVAL when T is NULL. */
int jp_two_path_filter(jp_ctx* ctx, const jp_rel* R, const jp_rel* S, const jp_rel* T,
                       jp_result* out);

/* Orders of jp_two_path_counts. */
#define JP_ORDER_PAIRS  0    /* (x, z) ascending as signed int32 */
#define JP_ORDER_COUNT  1    /* count descending; equal counts in (x, z) order */

/* Set similarity join with witness counts (Section 1 "Set Similarity"; its ordered form,
 * Section 4 "Ordered SSJ"): every pair (a, c) whose sets R(a, .) and S(c, .) share at least
 * c_min values of y, with that number -- the entry M_ac of the product M1 x M2 of Section 2.2
 * (c_min = 1 gives the two-path query with its counts).  The pairs a = c are included for a
 * self-join, as the definition has them.  Algorithm 1's split is kept (the context's threshold
 * mode): the heavy product's entries are read from the tensor cores' FP32 accumulators (exact
 * below 2^24 shared values), the light witnesses are counted by sorting each x's light
 * candidates, and the two counts of a pair are added.
 *   S      NULL means S = R;
 *   c_min  >= 1;
 *   order  JP_ORDER_PAIRS or JP_ORDER_COUNT;
 *   out    k = 3: col[0] = x, col[1] = z, col[2] = count (int32).
 * A heavy part with 2^24 or more heavy y gives JP_EUNSUPPORTED (its counts could pass the
 * FP32 accumulators' exact range; choose larger thresholds).
 * Memory: the heavy count matrix (4 bytes per heavy x and heavy z pair; JP_EUNSUPPORTED above
 * 64 GiB) and the light candidates of a range of x at a time (jp_set_count_chunk); one x with
 * 2^31 or more light candidates, or 2^32 or more result pairs, gives JP_EUNSUPPORTED.  Other
 * errors as jp_two_path. */
int jp_two_path_counts(jp_ctx* ctx, const jp_rel* R, const jp_rel* S, int64_t c_min, int order,
                       jp_result* out);

/* Light candidates jp_two_path_counts sorts in one pass (default 2^27; a pass takes 40 bytes of
 * workspace per candidate).  A smaller value bounds memory at the cost of more passes. */
int jp_set_count_chunk(jp_ctx* ctx, int64_t candidates);

/* Star query Q*_k (Section 2.1, Section 3.2) over rels[0..k-1], 2 <= k <= 8;
 * on success *out holds the sorted distinct k-tuples (k columns).  k = 2 is the two-path
 * query with S = rels[1]; k = 3 runs the Section 3.2 algorithm factorised on (x1, x2); for
 * k > 3 the relations R3..Rk are first grouped on y into one relation whose x is the id of a
 * distinct tuple (a3, .., ak) sharing a y (JP_EUNSUPPORTED if that relation would hold 2^31
 * or more tuples), the k = 3 algorithm runs on (R1, R2, it), and the ids are expanded. */
int jp_star(jp_ctx* ctx, int k, const jp_rel* rels, jp_result* out);

/* Batch of star queries Q*_3 (Section 3.2) in one pass of the star pipeline: query q is
 * Q*_3(R1_q, R2_q, R3_q).  Every x_i and every y is tagged with its query and
 * dictionary-encoded (y over the three relations together), so the batch is the single star
 * query of the tagged union: no witness joins tuples of two queries.
 *   rels     three relations; relation i holds the queries' tuples one after another;
 *   qoff     host, 3 x (nq + 1) entries: query q's tuples of relation i are
 *            [qoff[i (nq+1) + q], qoff[i (nq+1) + q + 1]); each row starts at 0, ends at
 *            rels[i].n and does not decrease (empty queries are allowed);
 *   out      one result (k = 3) holding the queries' sorted distinct triples, query after
 *            query;
 *   out_off  host, nq + 1 entries, receives where each query's triples start.
 * Thresholds by the context's mode for the union.  Errors as jp_star; JP_EINVAL for bad
 * offsets. */
int jp_star_batch(jp_ctx* ctx, int32_t nq, const jp_rel* rels, const int64_t* qoff,
                  jp_result* out, int64_t* out_off);

/* Statistics of the last successful query. */
int jp_get_stats(const jp_ctx* ctx, jp_stats* stats);

/* Copy result columns to host buffers host_cols[0..k-1] (each >= count
 * entries; pinned memory is fastest) and wait for the copy. */
int jp_result_to_host(jp_ctx* ctx, const jp_result* res, int32_t* const* host_cols);

/* Return a result's device memory (stream-ordered) and zero *res. */
void jp_result_free(jp_ctx* ctx, jp_result* res);

/* Message of the last failed call on this context ("" if none). */
const char* jp_last_error(const jp_ctx* ctx);

/* ---- Learned threshold predictor ----
 * The paper chooses Delta1, Delta2 with a cost model whose constants are
 * measured by hand (Section 5, Table 2, Algorithm 3).  The predictor learns the
 * choice instead: a network maps a relation's degree distribution to
 * (ln Delta1, ln Delta2), trained on the thresholds that timed best on the
 * GPU.  Features: two 64-bin histograms (x degrees; y degrees taken as
 * max(deg_R(y), deg_S(y))) with bin(d) = min(63, floor(4 log2 d)) computed
 * with integers; a bin holding c values enters as log2(1 + c) / 32, so the
 * features carry the relation's size as well as its degree law.
 * Network: 128 -> 256 -> 256 -> 2 with
 * ReLU, weights used in bfloat16, products and sums in float32, float32
 * master weights updated by Adam.  Parameters are one float array of
 * JP_MLP_PARAMS entries: W1[128][256], b1[256], W2[256][256], b2[256],
 * W3[256][2], b3[2] (W[i][j] maps input i to output j). */
#define JP_MLP_PARAMS 99330
#define JP_MLP_MAX_BATCH 1024
typedef struct jp_mlp jp_mlp;

/* The 128 features of the query jp_two_path(ctx, R, S) would run (host out). */
int jp_features(jp_ctx* ctx, const jp_rel* R, const jp_rel* S, float* out128);

/* Model used by JP_LEARNED (borrowed: it must outlive its use; NULL clears). */
int jp_set_predictor(jp_ctx* ctx, jp_mlp* model);

/* Create a model on `device`, working on `stream`; parameters start at zero. */
int jp_mlp_create(jp_mlp** model, int device, void* stream);
void jp_mlp_destroy(jp_mlp* model);
/* Copy the float32 master parameters in or out (host arrays of n entries,
 * n == JP_MLP_PARAMS); setting them also resets the Adam state. */
int jp_mlp_set_params(jp_mlp* model, const float* params, int64_t n);
int jp_mlp_get_params(jp_mlp* model, float* params, int64_t n);
/* Forward pass: X[B][128] host in, Y[B][2] host out, 1 <= B <= JP_MLP_MAX_BATCH. */
int jp_mlp_forward(jp_mlp* model, const float* X, int B, float* Y);
/* Gradients of the loss mean_b ||Y_b - T_b||^2 w.r.t. all parameters
 * (host array of JP_MLP_PARAMS, may be NULL) and the loss (host, may be NULL). */
int jp_mlp_gradients(jp_mlp* model, const float* X, const float* T, int B, float* grad,
                     float* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr on
 * the batch; *loss (host, may be NULL) gets the loss before the step. */
int jp_mlp_train_step(jp_mlp* model, const float* X, const float* T, int B, float lr,
                      float* loss);

/* ---- Allocation-free two-path query (the paper has no counterpart) ----
 * For callers that cannot allocate device memory when they query: services
 * that reserve their whole device-memory budget at start-up and forbid later
 * allocations (one more allocation would fail or fragment that budget),
 * plug-ins inside a host program that owns every device allocation and gives
 * its extensions none, and latency-bound loops for which an allocation, which
 * can wait for the device, costs more than the query.  It runs the
 * jp_two_path pipeline with every scratch buffer carved from one static
 * __device__ array of JP_NOALLOC_SCRATCH_BYTES (held by every GPU that loads
 * the library until the process exits) and writes into the caller's buffers.
 * It calls no cudaMalloc, cudaFree or other allocating routine and needs no
 * jp_ctx.
 *  - R, S: DEVICE pointers only (host pointers: JP_EINVAL); S == NULL means
 *    S = R.  Each relation holds at most JP_NOALLOC_MAX_TUPLES tuples
 *    (larger: JP_EUNSUPPORTED, checked before any work).
 *  - mode: JP_FIXED (delta1, delta2 >= 1) or JP_CLOSED_FORM; other modes are
 *    rejected with JP_EINVAL.
 *  - out_x, out_z: device buffers of out_cap entries each.  *out_count (a
 *    host pointer) receives the number of result pairs; when it exceeds
 *    out_cap nothing is written and JP_EOVERFLOW is returned, so the caller
 *    can retry with larger buffers.  Output order and content are those of
 *    jp_two_path.
 *  - A query whose scratch does not fit in the array fails with
 *    JP_EUNSUPPORTED.
 *  - Work runs on `stream` (a cudaStream_t) on the current device; the call
 *    returns once its work on the stream has finished, on success and on
 *    failure.  The first call on a device looks up the array's device address
 *    with cudaGetSymbolAddress.
 *  - Every call shares the array, which keeps the last call's contents; the
 *    call itself clears whatever must start at zero.  Calls that overlap on
 *    the GPU (from several host threads or streams) race on the array: the
 *    caller must serialise them. */
#define JP_NOALLOC_SCRATCH_BYTES (128u << 20)
#define JP_NOALLOC_MAX_TUPLES    (1 << 19)
int jp_two_path_noalloc(const jp_rel* R, const jp_rel* S, int mode, int64_t delta1,
                        int64_t delta2, int32_t* out_x, int32_t* out_z, int64_t out_cap,
                        int64_t* out_count, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* JP_H */
