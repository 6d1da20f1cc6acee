// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/jp.h"

namespace jp {

// ---------------------------------------------------------------- errors
struct Error {
    int code;
    std::string msg;
};

#define JP_CUDA_TRY(expr)                                                              \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess)                                                         \
            throw ::jp::Error{JP_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

// Every kernel launch of the library is followed by JP_CHECK_LAUNCH, which
// also counts it (reported per query in jp_stats.kernel_launches).  The
// counter is per host thread: a call runs on its caller's thread, so calls
// made from other threads at the same time do not mix their counts.
extern thread_local int64_t g_launches;
#define JP_CHECK_LAUNCH()                 \
    do {                                  \
        ++::jp::g_launches;               \
        JP_CUDA_TRY(cudaGetLastError());  \
    } while (0)

// Device status word bits (set by kernels; read by the host at sync points).
enum : uint32_t {
    ST_OVERFLOW = 1u << 0,   // a capacity check failed and the write was skipped
    ST_TIMEOUT = 1u << 1,    // a bounded wait ran out
    ST_BADINDEX = 1u << 2,   // an index check failed (should never happen)
};

// ---------------------------------------------------------------- memory
// Workspace: chunks obtained through the context's allocator, carved by a
// bump pointer that is reset at the start of every query and reused.
struct Arena {
    struct Chunk { char* p; size_t size; };
    std::vector<Chunk> chunks;
    size_t cur = 0;      // chunk index
    size_t off = 0;      // offset in chunk
    jp_alloc_fn alloc = nullptr;
    jp_free_fn release = nullptr;
    void* user = nullptr;
    cudaStream_t stream = nullptr;
    size_t peak = 0, used = 0;
    size_t hint = 0;     // size of the next chunk to allocate (the last query's peak)

    void reset() { cur = 0; off = 0; used = 0; }
    // Start of a query: give the chunks back when they hold more than three
    // times what the previous query used, so that one large query does not
    // pin its workspace for the context's lifetime.
    void begin();
    void* raw_alloc(size_t bytes);
    void raw_free(void* p, size_t bytes);
    void* carve(size_t bytes);
    void release_all();
    template <class T> T* get(size_t count) {
        return reinterpret_cast<T*>(carve(count * sizeof(T) + 16));
    }
};

// ---------------------------------------------------------------- primitives
// Exclusive scan of n values into out (may alias in); writes the total to
// *d_total if non-null (device pointer).
void scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* d_total, Arena& ws,
              cudaStream_t st);
void scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* d_total, Arena& ws,
              cudaStream_t st);

// LSD radix sort of uint64 keys.  Sorts keys[0..n) (using tmp as the ping-pong
// buffer) and returns whichever of the two buffers holds the sorted keys.
// Byte passes whose digit is constant over all keys are skipped; this needs
// one host synchronisation (the 8x256 digit histogram).  The buffer pair
// hist_host (pinned, >= 2048 entries) receives the histogram.
uint64_t* radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, Arena& ws, cudaStream_t st,
                         uint32_t* hist_host);

// Compact the distinct entries of sorted keys into out; count to *d_count.
void unique_u64(const uint64_t* keys, int64_t n, uint64_t* out, uint32_t* d_count, Arena& ws,
                cudaStream_t st);

// ---------------------------------------------------------------- pipeline state
// Normalised relations in dense ids.  All arrays are device memory.
struct Graph {
    bool self = true;
    int64_t nr = 0, ns = 0;        // distinct tuples of R (after dropping dangling) and S
    int64_t nx = 0, ny = 0, nz = 0;
    int32_t* xval = nullptr;       // [nx] x id -> value
    int32_t* zval = nullptr;       // [nz] z id -> value (== xval for self-join)
    int32_t* yval = nullptr;       // [ny]
    int32_t* rxoff = nullptr;      // [nx+1] CSR of R by x
    int32_t* rycol = nullptr;      // [nr] y ids, sorted within a row
    int32_t* syoff = nullptr;      // [ny+1] CSR of S by y
    int32_t* szcol = nullptr;      // [ns] z ids, sorted within a row
    int32_t* deg_rx = nullptr;     // [nx]
    int32_t* deg_ry = nullptr;     // [ny]
    int32_t* deg_sy = nullptr;     // [ny]
    int32_t* deg_sz = nullptr;     // [nz]
    int64_t* xsum = nullptr;       // [nx] sum over x's y of deg_S(y): x's join candidates (may be null)
    double out_join = 0;
};

struct Partition {
    int64_t d1 = 1, d2 = 1;
    int64_t u = 0, v = 0, w = 0;
    int32_t* hx = nullptr;      // [nx] heavy x index or -1
    int32_t* hy = nullptr;      // [ny]
    int32_t* hz = nullptr;      // [nz]
    int32_t* hx_inv = nullptr;  // [u]
    int32_t* hy_inv = nullptr;  // [v]
    int32_t* hz_inv = nullptr;  // [w]
    int32_t* sloff = nullptr;   // [v+1] light-z lists of heavy y (S^- restricted to heavy y)
    int32_t* slcol = nullptr;
};

struct Heavy {
    int64_t u_pad = 0, v_pad = 0, w_pad = 0;
    uint8_t* A = nullptr;       // [u_pad][v_pad] 0x00 / 0x38 (FP8 E4M3 0.0 / 1.0)
    uint8_t* B = nullptr;       // [w_pad][v_pad]
    uint32_t* G = nullptr;      // [u_pad][g_stride] bit (h,c) = product (h,c) > 0
    int64_t g_stride = 0;       // words per row
    int tbn = 256;              // product tile width (rows of B per CTA): 128 or 256
    bool present = false;
};

// Builders (jp_build.cu)
void build_graph(const jp_rel* R, const jp_rel* S, Graph& g, Arena& ws, cudaStream_t st,
                 uint32_t* d_status, uint32_t* hist_host, int64_t* host_scalars);

// Batches: for every tile of the heavy product, the range of K blocks [x, y)
// shared by the queries of its rows and of its columns (empty when they share
// none: the heavy block of a batch is block-diagonal by query).
int2* batch_tile_ranges(const Partition& p, const Heavy& h, const int32_t* xq_begin,
                        const int32_t* yq_begin, int32_t nq, Arena& ws, cudaStream_t st);

// Measured dense tensor rates (TFLOP/s): tcgen05 FP8 MMAs of the product's
// shape on shared-memory operands, and legacy INT8 mma.sync m16n8k32.
void measure_peaks(int sms, double* fp8_tflops, double* int8_tflops, uint32_t* d_status,
                   Arena& ws, cudaStream_t st);

// A kernel whose bounded wait (the heavy product's) is made to run out after ns.
void wait_selftest(uint32_t* d_status, int64_t ns, cudaStream_t st);

// Batches of self-joins (jp_batch.cu): global ids of (query, value) pairs.
struct BatchIds {
    int32_t* xg = nullptr;        // [n] global x id of every tuple
    int32_t* yg = nullptr;        // [n] global y id of every tuple
    int32_t* xorig = nullptr;     // [nxg] global x id -> value
    int64_t nxg = 0;
    int32_t* xq_begin = nullptr;  // [nq + 1] first global x id of every query (nxg at nq)
    int32_t* yq_begin = nullptr;  // [nq + 1] first global y id of every query
};
void batch_encode(const int32_t* x, const int32_t* y, int64_t n, int32_t nq,
                  const int64_t* qoff_host, BatchIds& b, Arena& ws, cudaStream_t st,
                  uint32_t* hist_host, uint32_t* d_status);
// Batches of star queries k = 3 (jp_batch.cu): each relation's x tagged and
// encoded, y encoded over the three relations together.
struct StarBatchIds {
    jp_rel rel[3] = {};               // the relations in global ids
    int32_t* xorig[3] = {};           // global x_i id -> value
    int32_t* x1q_begin = nullptr;     // [nq + 1] first global x1 id of every query
};
void star_batch_encode(const jp_rel* rels, int32_t nq, const int64_t* qoff_host, StarBatchIds& b,
                       Arena& ws, cudaStream_t st, uint32_t* hist_host, uint32_t* d_status);
// Output offset of every query's first triple (host, nq + 1 entries), then the
// three columns mapped from global ids to values in place.
void star_batch_finish(int32_t* const* cols, int64_t count, const StarBatchIds& b, int32_t nq,
                       int64_t* host_offsets, Arena& ws, cudaStream_t st);
// Output offset of every query's first pair (host, nq + 1 entries).
void batch_offsets(const int64_t* out_off, int64_t nx, int64_t count, const BatchIds& b,
                   int32_t nq, int64_t* host_offsets, Arena& ws, cudaStream_t st);

// Boolean set intersection in batches (jp_filter.cu, Section 3.3): the
// candidate pairs T and R, S reduced to T's x and z values.
struct FilterState {
    uint64_t* tkeys = nullptr;    // [nt] sorted distinct pairs of T, (x ^ 2^31) << 32 | (z ^ 2^31)
    int64_t nt = 0;
    jp_rel R{}, S{};              // R restricted to T's x values, S to T's z values
    uint32_t* flag = nullptr;     // [nt] pair found in the query's output (filter_find)
    uint32_t* pos = nullptr;      // [nt] exclusive scan of flag
};
void filter_reduce(const jp_rel& R, const jp_rel& S, const jp_rel& T, FilterState& fs, Arena& ws,
                   cudaStream_t st, uint32_t* hist_host);
// Marks the pairs of T present in the sorted output (ox, oz)[0..no); returns how many.
int64_t filter_find(FilterState& fs, const int32_t* ox, const int32_t* oz, int64_t no, Arena& ws,
                    cudaStream_t st);
// Writes the marked pairs, in order, to (px, pz).
void filter_emit(const FilterState& fs, int32_t* px, int32_t* pz, cudaStream_t st);

// Threshold selection (jp_select.cu)
double out_estimate(double dom_x, double out_join, double N);
// *judged (JP_LEARNED): 1 the model's thresholds kept, 2 replaced by Algorithm 3's.
jp_cost_model default_cost_model();
bool valid_cost_model(const jp_cost_model& K);
void select_thresholds(const Graph& g, int mode, int64_t fd1, int64_t fd2, int64_t* d1,
                       int64_t* d2, double* out_est, Arena& ws, cudaStream_t st,
                       const jp_cost_model& K, jp_mlp* predictor = nullptr,
                       int* judged = nullptr);

// Learned predictor (jp_mlp.cu): the 128 degree features of a built graph and
// the thresholds a model predicts for them.
void graph_features(const Graph& g, float* host128, Arena& ws, cudaStream_t st);
void mlp_predict(jp_mlp* model, const float* host128, int64_t N, int64_t* d1, int64_t* d2);

// Partition (jp_partition.cu)
void build_partition(const Graph& g, Partition& p, Arena& ws, cudaStream_t st,
                     int64_t* host_scalars);
// h[i] = rank among values with max(deg_a, deg_b) > thr, else -1; returns the count
int64_t heavy_ids(const int32_t* deg_a, const int32_t* deg_b, int64_t n, int64_t thr,
                  int32_t* h, int32_t* h_inv, Arena& ws, cudaStream_t st);
// light-z lists (z with hz < 0) of the heavy y values of a CSR by y
void build_light_z_lists(const int32_t* syoff, const int32_t* szcol, Partition& p, Arena& ws,
                         cudaStream_t st);

// Heavy part (jp_gemm.cu)
void heavy_pack(const Graph& g, const Partition& p, Heavy& h, Arena& ws, cudaStream_t st);
// Product tile width for a heavy block: width 128 or 256 as given, or 0
// (auto): 128 when the block has at most auto_max_tiles tiles of 128 x 256.
int pick_tile(const Heavy& h, int width, int64_t auto_max_tiles);
// tiles: null, or (batches) the K-block range of every tile (batch_tile_ranges,
// computed for h.tbn).
void heavy_gemm(Heavy& h, const Partition& p, uint32_t* d_status, cudaStream_t st,
                const int2* tiles = nullptr);
// The heavy product's entries (witness counts) as uint32 into C[u_pad][w_pad].
void heavy_gemm_counts(const Heavy& h, uint32_t* C, uint32_t* d_status, cudaStream_t st);

// Witness counts and the set similarity join (jp_counts.cu): the pairs with
// M_ac >= c_min as (x, z, count) columns in the workspace, in (x, z) order or
// by decreasing count.  Returns the number of pairs and the light candidates.
struct CountResult {
    int32_t* x = nullptr;
    int32_t* z = nullptr;
    int32_t* cnt = nullptr;
    int64_t n = 0;
    int64_t candidates = 0;
    double ms_fill = 0, ms_sort = 0, ms_merge = 0;   // device ms summed over the x ranges
    int64_t ranges = 0;
    int64_t light_pairs = 0;     // distinct (x, z) among the light candidates
    int64_t heavy_pairs = 0;     // nonzero entries of the heavy product
};
void count_pairs(const Graph& g, const Partition& p, const Heavy& h, int64_t c_min, int order,
                 CountResult& out, Arena& ws, cudaStream_t st, uint32_t* d_status,
                 uint32_t* hist_host, int64_t chunk_candidates);

// Light part + union (jp_light.cu)
// A row's list: tmp_off >= 0 is its offset in tmp, holding z values, or, with
// TMP_IDS set, z ids (bitmap rows); tmp_off < 0 is -(offset in szval) - 1 for
// a row with a single neighbour list, read in place.
constexpr int64_t TMP_IDS = (int64_t)1 << 62;

struct LightResult {
    int64_t* tmp_off = nullptr;   // [nx]
    int32_t* szval = nullptr;     // [ns] zval[szcol]
    int32_t* cnt = nullptr;       // [nx]
    int32_t* tmp = nullptr;
    int64_t tmp_cap = 0;
    int64_t candidates = 0;
    // per class: warp sort, bucket sort, single-list copy, bitmap, merge 4096, merge 8192, hubs,
    // merge 2048
    int64_t class_x[8] = {};      // x values
    int64_t class_cand[8] = {};   // candidates
    int64_t class_deg[8] = {};    // neighbour entries
    int32_t* tile_x = nullptr;             // x holding the first output of each output tile
};
// qbeg/nq: for batches, the first x id of every query (nq + 1 entries), which
// bounds the z range of a row; null otherwise.
void light_and_union(const Graph& g, const Partition& p, const Heavy& h, LightResult& lr,
                     Arena& ws, cudaStream_t st, uint32_t* d_status, int64_t* host_scalars,
                     const int32_t* qbeg = nullptr, int32_t nq = 0);

// Output (jp_output.cu)
int64_t output_count(const Graph& g, LightResult& lr, int64_t* out_off, Arena& ws,
                     cudaStream_t st, int64_t* host_scalars);
void output_write(const Graph& g, const LightResult& lr, const int64_t* out_off, int64_t count,
                  int32_t* out_x, int32_t* out_z, cudaStream_t st);
// Same placement with one or two per-row value columns (rowval2 may be NULL):
// output o of row r gets (rowval[r], rowval2[r], zval[list entry]).
void output_write_rows(const Graph& g, const LightResult& lr, const int64_t* out_off,
                       int64_t count, const int32_t* rowval, const int32_t* rowval2,
                       int32_t* out_row, int32_t* out_row2, int32_t* out_z, cudaStream_t st);
// Two-path output whose x and z values are ids into vmap (batches: global id -> value).
void output_write_mapped(const Graph& g, const LightResult& lr, const int64_t* out_off,
                         int64_t count, const int32_t* vmap, int32_t* out_x, int32_t* out_z,
                         cudaStream_t st);

// Star query k = 3 (jp_star.cu): builds the virtual two-path instance whose
// rows are the (x1, x2) pairs, whose neighbour lists are the shared y of each
// pair and whose S is R3 indexed by y; row1/row2 hold each row's x1/x2 value.
struct StarOut {
    Graph g;
    Partition p;
    int32_t* row1 = nullptr;
    int32_t* row2 = nullptr;
    int64_t n_rel[3] = {0, 0, 0}, nx[3] = {0, 0, 0};
    int64_t ny = 0, triples = 0, groups = 0, d1 = 1, d2 = 1;
    double out_join = 0;   // full star join size sum_y d1(y) d2(y) d3(y)
};
void run_star3(const jp_rel* rels, int mode, int64_t fd1, int64_t fd2, StarOut& so, Arena& ws,
               cudaStream_t st, uint32_t* d_status, uint32_t* hist_host);
// Star queries with k > 3 (jp_star.cu): the tail relations grouped on y.
struct PairRel {
    int32_t* x = nullptr;   // [n] group id of every tuple
    int32_t* y = nullptr;   // [n] y value
    int64_t n = 0;
    int32_t* gp = nullptr;  // [ng] the pair's first value
    int32_t* gq = nullptr;  // [ng] the pair's second value (the next level's group id)
    int64_t ng = 0;
};
void pair_relation(const jp_rel* P, const jp_rel* Q, PairRel& out, Arena& ws, cudaStream_t st,
                   uint32_t* hist_host);
struct StarChain {
    int levels = 0;                 // k - 3
    const int32_t* gp[6] = {};
    const int32_t* gq[6] = {};
};
void star_expand(const int32_t* g3, int64_t n, const StarChain& chain, int32_t* const* cols_dev,
                 cudaStream_t st);
// Integer (Delta1, Delta2) minimising the Section 3.2 star cost on a log grid.
void star_thresholds(int64_t N, double out_est, int k, int64_t* d1, int64_t* d2);

// Small helpers
int grid_for(int64_t n, int block, int max_blocks = 152 * 32);

// Per-query device timing with CUDA events on the query stream, one
// begin/end pair per pass or kernel (reported in jp_stats.ms_pass).
enum TimerSlot {
    TM_BUILD = 0, TM_SELECT, TM_PARTITION, TM_PACK, TM_GEMM, TM_CLASSIFY, TM_LIGHT_WARP,
    TM_LIGHT_C2, TM_LIGHT_MERGE, TM_LIGHT_BITMAP, TM_COUNT, TM_PLACE, TM_TOTAL, TM_SLOTS = 16
};
struct Timer {
    cudaEvent_t b[TM_SLOTS] = {}, e[TM_SLOTS] = {};
    bool used[TM_SLOTS] = {};
    cudaStream_t st = nullptr;
    void begin(int k) { cudaEventRecord(b[k], st); used[k] = true; }
    void end(int k) { cudaEventRecord(e[k], st); }
    float ms(int k) const {
        float v = 0;
        if (used[k] && cudaEventElapsedTime(&v, b[k], e[k]) != cudaSuccess) { cudaGetLastError(); v = 0; }
        return v;
    }
};
// The timer of the call running on this host thread (null: none).
extern thread_local Timer* g_timer;

// Raise `func`'s dynamic shared-memory limit to `bytes` on the current
// device.  The attribute belongs to each device's context, so it is set once
// per (kernel, device) and again whenever a larger value is needed.
void smem_limit(const void* func, size_t bytes);
inline void tbegin(int k) { if (g_timer) g_timer->begin(k); }
inline void tend(int k) { if (g_timer) g_timer->end(k); }

}  // namespace jp
