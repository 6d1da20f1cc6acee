// C-ABI entry points: context, workspace, argument checks and the two-path
// pipeline of Algorithm 1 (Section 3.1):
//   index build -> thresholds -> partition -> heavy matrices + product ->
//   light expansion/deduplication + union -> output placement.
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>

#include "jp_internal.cuh"

struct jp_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    jp::Arena ws;
    int mode = JP_CLOSED_FORM;
    int64_t d1 = 1, d2 = 1;
    std::string err;
    jp_stats stats;
    bool have_stats = false;
    uint32_t* hist_host = nullptr;     // pinned, 2048 entries
    int64_t* host_scalars = nullptr;   // pinned, 64 entries
    uint32_t* d_status = nullptr;      // device status word
    jp::Timer tm;
    jp_mlp* predictor = nullptr;       // borrowed model for JP_LEARNED
    int64_t count_chunk = (int64_t)1 << 27;   // light candidates per pass of jp_two_path_counts
    jp_cost_model cost = jp::default_cost_model();   // Algorithm 3's constants
    int gemm_width = 0;                 // product tile width: 0 auto, 128 or 256
    int64_t gemm_auto_tiles = 32;       // auto: narrow tiles up to this many 128 x 256 tiles
                                        // (the crossover the tile autotuner measured on GB300)
};

namespace jp {

thread_local int64_t g_launches = 0;
thread_local Timer* g_timer = nullptr;

void smem_limit(const void* func, size_t bytes) {
    struct Entry { const void* f; int dev; size_t bytes; };
    static std::mutex mu;
    static std::vector<Entry> done;
    int dev = 0;
    JP_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    for (Entry& e : done)
        if (e.f == func && e.dev == dev) {
            if (e.bytes >= bytes) return;
            JP_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
            e.bytes = bytes;
            return;
        }
    JP_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    done.push_back({func, dev, bytes});
}

void* Arena::raw_alloc(size_t bytes) {
    if (alloc) return alloc(bytes, (void*)stream, user);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void Arena::raw_free(void* p, size_t bytes) {
    if (!p) return;
    if (release) release(p, bytes, (void*)stream, user);
    else cudaFreeAsync(p, stream);
}

void* Arena::carve(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    while (cur < chunks.size()) {
        if (off + bytes <= chunks[cur].size) {
            void* p = chunks[cur].p + off;
            off += bytes;
            used += bytes;
            if (used > peak) peak = used;
            return p;
        }
        ++cur;
        off = 0;
    }
    size_t total = 0;
    for (auto& c : chunks) total += c.size;
    size_t sz = bytes;
    if (sz < total) sz = total;
    if (sz < hint) sz = hint;
    hint = 0;
    if (sz < ((size_t)64 << 20)) sz = (size_t)64 << 20;
    void* p = raw_alloc(sz);
    if (!p) throw Error{JP_ENOMEM, "workspace allocation of " + std::to_string(sz) + " bytes failed"};
    chunks.push_back({reinterpret_cast<char*>(p), sz});
    cur = chunks.size() - 1;
    off = bytes;
    used += bytes;
    if (used > peak) peak = used;
    return p;
}

void Arena::begin() {
    size_t held = 0;
    for (auto& c : chunks) held += c.size;
    const size_t need = peak;
    // keep the chunks while they serve queries of this size (reallocating
    // them would fragment the allocator's pool); give them back when they
    // hold more than three times what the last query used
    if (held > ((size_t)1 << 30) && 3 * need < held) {
        release_all();
        hint = need;
    }
    reset();
    peak = 0;
}

void Arena::release_all() {
    for (auto& c : chunks) raw_free(c.p, c.size);
    chunks.clear();
    reset();
}

}  // namespace jp

namespace {

int fail(jp_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device copy of a relation (host inputs are copied into the workspace).
jp_rel to_device(jp_ctx* ctx, const jp_rel* r) {
    jp_rel d = *r;
    if (r->n == 0) return d;
    const size_t bytes = (size_t)r->n * sizeof(int32_t);
    if (!is_device_ptr(r->x)) {
        int32_t* p = ctx->ws.get<int32_t>(r->n);
        JP_CUDA_TRY(cudaMemcpyAsync(p, r->x, bytes, cudaMemcpyHostToDevice, ctx->stream));
        d.x = p;
    }
    if (!is_device_ptr(r->y)) {
        int32_t* p = ctx->ws.get<int32_t>(r->n);
        JP_CUDA_TRY(cudaMemcpyAsync(p, r->y, bytes, cudaMemcpyHostToDevice, ctx->stream));
        d.y = p;
    }
    return d;
}

int check_rel(jp_ctx* ctx, const jp_rel* r, const char* name) {
    if (!r) return fail(ctx, JP_EINVAL, std::string(name) + " is NULL");
    if (r->n < 0) return fail(ctx, JP_EINVAL, std::string(name) + "->n is negative");
    if (r->n > 0 && (!r->x || !r->y)) return fail(ctx, JP_EINVAL, std::string(name) + " has a NULL column");
    if (r->n >= ((int64_t)1 << 31)) return fail(ctx, JP_EUNSUPPORTED, std::string(name) + " has 2^31 or more tuples");
    return JP_OK;
}

void status_check(jp_ctx* ctx) {
    uint32_t s = 0;
    JP_CUDA_TRY(cudaMemcpyAsync(&s, ctx->d_status, sizeof(s), cudaMemcpyDeviceToHost, ctx->stream));
    JP_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (s & jp::ST_TIMEOUT) throw jp::Error{JP_ETIMEOUT, "a bounded device wait ran out"};
    if (s & jp::ST_OVERFLOW) throw jp::Error{JP_EOVERFLOW, "a device capacity check failed"};
    if (s & jp::ST_BADINDEX) throw jp::Error{JP_EOVERFLOW, "a device index check failed"};
}

}  // namespace

namespace {

struct BatchArgs {
    int32_t nq;
    const int64_t* qoff;     // host, nq + 1
    int64_t* out_off;        // host, nq + 1
};

// Caller-owned output columns (jp_two_path_into): device pointers, or host
// memory the kernels can write (pinned, or any host memory on a device with
// pageable memory access).
struct ExtOut {
    int32_t* x;
    int32_t* z;
    int64_t cap;
    int64_t* count;          // host: |OUT|
};

// The address kernels use for a caller's output buffer, or null when the GPU
// cannot write it.
int32_t* kernel_ptr(jp_ctx* ctx, int32_t* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
        return a.device == ctx->device ? p : nullptr;
    if (a.type == cudaMemoryTypeHost) return reinterpret_cast<int32_t*>(a.devicePointer);
    int pageable = 0;
    if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, ctx->device) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return pageable ? p : nullptr;
}

// The two-path pipeline.  With a batch, R holds the queries' tuples one after
// another (batch->qoff) and is a self-join per query; its values are first
// encoded to (query, value) ids, and the output maps them back.
//
// With a candidate set T (the Section 3.3 batch of boolean set intersection
// queries), R and S are first reduced to T's x and z values, the pipeline
// answers the reduced query into the workspace, and the result is the pairs of
// T found in that output.
int run_two_path(jp_ctx* ctx, const jp_rel* R, const jp_rel* S, jp_result* out,
                 const BatchArgs* batch, const jp_rel* T = nullptr, const ExtOut* ext = nullptr) {
    if (!ctx) return JP_EINVAL;
    if (!out) return fail(ctx, JP_EINVAL, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    out->k = 2;
    int rc = check_rel(ctx, R, "R");
    if (rc) return rc;
    if (S && (rc = check_rel(ctx, S, "S"))) return rc;
    if (S && R->n + S->n >= ((int64_t)1 << 31)) return fail(ctx, JP_EUNSUPPORTED, "R and S together hold 2^31 or more tuples");
    if (T && (rc = check_rel(ctx, T, "T"))) return rc;
    const auto t_start = std::chrono::steady_clock::now();
    void* block = nullptr;
    size_t block_bytes = 0;
    try {
        JP_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = ctx->stream;
        ctx->ws.begin();
        const int64_t launches0 = jp::g_launches;
        JP_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), st));
        for (int i = 0; i < jp::TM_SLOTS; ++i) ctx->tm.used[i] = false;
        ctx->tm.st = st;
        jp::g_timer = &ctx->tm;
        ctx->tm.begin(jp::TM_TOTAL);
        jp_rel Rd = to_device(ctx, R);
        jp_rel Sd;
        if (S) Sd = to_device(ctx, S);
        jp::FilterState fs;
        if (T) {
            const jp_rel Td = to_device(ctx, T);
            jp::filter_reduce(Rd, S ? Sd : Rd, Td, fs, ctx->ws, st, ctx->hist_host);
            Rd = fs.R;
            Sd = fs.S;
        }
        const bool self = !T && ((S == nullptr) || (S->x == R->x && S->y == R->y && S->n == R->n));
        jp::BatchIds bid;
        if (batch) {
            jp::batch_encode(Rd.x, Rd.y, Rd.n, batch->nq, batch->qoff, bid, ctx->ws, st,
                             ctx->hist_host, ctx->d_status);
            Rd.x = bid.xg;
            Rd.y = bid.yg;
        }

        jp::Graph g;
        ctx->tm.begin(jp::TM_BUILD);
        jp::build_graph(&Rd, self ? nullptr : &Sd, g, ctx->ws, st, ctx->d_status, ctx->hist_host,
                        ctx->host_scalars);
        ctx->tm.end(jp::TM_BUILD);

        jp::Partition p;
        double out_est = 0;
        ctx->tm.begin(jp::TM_SELECT);
        int judged = 0;
        jp::select_thresholds(g, ctx->mode, ctx->d1, ctx->d2, &p.d1, &p.d2, &out_est, ctx->ws, st,
                              ctx->cost, ctx->predictor, &judged);
        ctx->tm.end(jp::TM_SELECT);
        ctx->tm.begin(jp::TM_PARTITION);
        jp::build_partition(g, p, ctx->ws, st, ctx->host_scalars);
        ctx->tm.end(jp::TM_PARTITION);

        jp::Heavy h;
        ctx->tm.begin(jp::TM_PACK);
        jp::heavy_pack(g, p, h, ctx->ws, st);
        h.tbn = jp::pick_tile(h, ctx->gemm_width, ctx->gemm_auto_tiles);
        ctx->tm.end(jp::TM_PACK);
        const int2* tiles = batch ? jp::batch_tile_ranges(p, h, bid.xq_begin, bid.yq_begin,
                                                          batch->nq, ctx->ws, st)
                                  : nullptr;
        jp::heavy_gemm(h, p, ctx->d_status, st, tiles);

        jp::LightResult lr;
        jp::light_and_union(g, p, h, lr, ctx->ws, st, ctx->d_status, ctx->host_scalars,
                            batch ? bid.xq_begin : nullptr, batch ? batch->nq : 0);

        int64_t* out_off = ctx->ws.get<int64_t>(g.nx + 1);
        ctx->tm.begin(jp::TM_COUNT);
        const int64_t count = jp::output_count(g, lr, out_off, ctx->ws, st, ctx->host_scalars);
        ctx->tm.end(jp::TM_COUNT);
        status_check(ctx);
        int64_t result_count = count;
        if (T) {
            int32_t* qx = ctx->ws.get<int32_t>(count + 1);
            int32_t* qz = ctx->ws.get<int32_t>(count + 1);
            ctx->tm.begin(jp::TM_PLACE);
            if (count > 0) jp::output_write(g, lr, out_off, count, qx, qz, st);
            ctx->tm.end(jp::TM_PLACE);
            result_count = jp::filter_find(fs, qx, qz, count, ctx->ws, st);
        }
        if (ext) {
            *ext->count = result_count;
            if (result_count > ext->cap)
                throw jp::Error{JP_EOVERFLOW, "the result has " + std::to_string(result_count) +
                                                  " pairs, more than the buffers hold"};
            if (result_count > 0) {
                int32_t* kx = kernel_ptr(ctx, ext->x);
                int32_t* kz = kernel_ptr(ctx, ext->z);
                if (!kx || !kz) throw jp::Error{JP_EINVAL, "an output buffer is not writable by the GPU"};
                ctx->tm.begin(jp::TM_PLACE);
                jp::output_write(g, lr, out_off, count, kx, kz, st);
                ctx->tm.end(jp::TM_PLACE);
            }
        } else if (result_count > 0) {
            block_bytes = (size_t)result_count * 2 * sizeof(int32_t) + 512;
            block = ctx->ws.raw_alloc(block_bytes);
            if (!block) throw jp::Error{JP_ENOMEM, "result allocation failed"};
            int32_t* ox = reinterpret_cast<int32_t*>(block);
            int32_t* oz = reinterpret_cast<int32_t*>(
                reinterpret_cast<char*>(block) + (((size_t)result_count * sizeof(int32_t) + 255) & ~(size_t)255));
            if (!T) ctx->tm.begin(jp::TM_PLACE);
            if (T)
                jp::filter_emit(fs, ox, oz, st);
            else if (batch)
                jp::output_write_mapped(g, lr, out_off, count, bid.xorig, ox, oz, st);
            else
                jp::output_write(g, lr, out_off, count, ox, oz, st);
            if (!T) ctx->tm.end(jp::TM_PLACE);
            out->col[0] = ox;
            out->col[1] = oz;
        }
        if (batch) jp::batch_offsets(out_off, g.nx, count, bid, batch->nq, batch->out_off, ctx->ws, st);
        ctx->tm.end(jp::TM_TOTAL);
        status_check(ctx);
        jp::g_timer = nullptr;
        out->count = result_count;
        out->_block = block;
        out->_bytes = block_bytes;

        jp_stats& s = ctx->stats;
        std::memset(&s, 0, sizeof(s));
        s.n_r = g.nr;
        s.n_s = g.ns;
        s.dom_x = g.nx;
        s.dom_y = g.ny;
        s.dom_z = g.nz;
        s.out_join = g.out_join;
        s.out_estimate = out_est;
        s.delta1 = p.d1;
        s.delta2 = p.d2;
        s.threshold_mode = ctx->mode;
        s.u = p.u;
        s.v = p.v;
        s.w = p.w;
        s.light_candidates = lr.candidates;
        s.out_count = result_count;
        s.learned_judged = judged;
        s.filter_pairs = T ? fs.nt : 0;
        s.filter_query_out = T ? count : 0;
        s.kernel_launches = jp::g_launches - launches0;
        s.gemm_tile = h.present ? h.tbn : 0;
        for (int q = 0; q < 8; ++q) {
            s.light_x[q] = lr.class_x[q];
            s.light_cand[q] = lr.class_cand[q];
            s.light_deg[q] = lr.class_deg[q];
        }
        for (int i = 0; i < jp::TM_SLOTS; ++i) s.ms_pass[i] = ctx->tm.ms(i);
        s.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        ctx->have_stats = true;
        ctx->err.clear();
        return JP_OK;
    } catch (const jp::Error& e) {
        jp::g_timer = nullptr;
        if (block) ctx->ws.raw_free(block, block_bytes);
        std::memset(out, 0, sizeof(*out));
        return fail(ctx, e.code, e.msg);
    } catch (const std::bad_alloc&) {
        if (block) ctx->ws.raw_free(block, block_bytes);
        std::memset(out, 0, sizeof(*out));
        return fail(ctx, JP_ENOMEM, "host allocation failed");
    }
}

}  // namespace

extern "C" {

int jp_create(jp_ctx** out, int device, void* stream, jp_alloc_fn alloc, jp_free_fn release,
              void* user) {
    if (!out) return JP_EINVAL;
    *out = nullptr;
    if ((alloc == nullptr) != (release == nullptr)) return JP_EINVAL;
    jp_ctx* ctx = new (std::nothrow) jp_ctx();
    if (!ctx) return JP_ENOMEM;
    try {
        int ndev = 0;
        JP_CUDA_TRY(cudaGetDeviceCount(&ndev));
        if (device < 0 || device >= ndev) throw jp::Error{JP_EINVAL, "no such device"};
        cudaDeviceProp prop;
        JP_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
        if (!(prop.major == 10 && prop.minor == 3))
            throw jp::Error{JP_EUNSUPPORTED, "device is not compute capability 10.3 (sm_103)"};
        JP_CUDA_TRY(cudaSetDevice(device));
        ctx->device = device;
        ctx->stream = (cudaStream_t)stream;
        ctx->ws.alloc = alloc;
        ctx->ws.release = release;
        ctx->ws.user = user;
        ctx->ws.stream = ctx->stream;
        JP_CUDA_TRY(cudaHostAlloc((void**)&ctx->hist_host, 2048 * sizeof(uint32_t), cudaHostAllocDefault));
        JP_CUDA_TRY(cudaHostAlloc((void**)&ctx->host_scalars, 64 * sizeof(int64_t), cudaHostAllocDefault));
        JP_CUDA_TRY(cudaMalloc((void**)&ctx->d_status, 256));
        for (int i = 0; i < jp::TM_SLOTS; ++i) {
            JP_CUDA_TRY(cudaEventCreate(&ctx->tm.b[i]));
            JP_CUDA_TRY(cudaEventCreate(&ctx->tm.e[i]));
        }
        std::memset(&ctx->stats, 0, sizeof(ctx->stats));
    } catch (const jp::Error& e) {
        int code = e.code;
        jp_destroy(ctx);
        return code;
    }
    *out = ctx;
    return JP_OK;
}

void jp_destroy(jp_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream || true) cudaStreamSynchronize(ctx->stream);
    ctx->ws.release_all();
    cudaStreamSynchronize(ctx->stream);
    if (ctx->hist_host) cudaFreeHost(ctx->hist_host);
    if (ctx->host_scalars) cudaFreeHost(ctx->host_scalars);
    if (ctx->d_status) cudaFree(ctx->d_status);
    for (int i = 0; i < jp::TM_SLOTS; ++i) {
        if (ctx->tm.b[i]) cudaEventDestroy(ctx->tm.b[i]);
        if (ctx->tm.e[i]) cudaEventDestroy(ctx->tm.e[i]);
    }
    cudaGetLastError();
    delete ctx;
}

int jp_set_threshold(jp_ctx* ctx, int mode, int64_t delta1, int64_t delta2) {
    if (!ctx) return JP_EINVAL;
    if (mode != JP_FIXED && mode != JP_CLOSED_FORM && mode != JP_COST_MODEL && mode != JP_LEARNED)
        return fail(ctx, JP_EINVAL, "unknown threshold mode");
    if (mode == JP_FIXED && (delta1 < 1 || delta2 < 1))
        return fail(ctx, JP_EINVAL, "thresholds must be >= 1");
    ctx->mode = mode;
    ctx->d1 = delta1;
    ctx->d2 = delta2;
    return JP_OK;
}

int jp_set_cost_model(jp_ctx* ctx, const jp_cost_model* model) {
    if (!ctx) return JP_EINVAL;
    if (!model) {
        ctx->cost = jp::default_cost_model();
        return JP_OK;
    }
    if (!jp::valid_cost_model(*model)) return fail(ctx, JP_EINVAL, "cost model constant out of range");
    ctx->cost = *model;
    return JP_OK;
}

int jp_get_cost_model(const jp_ctx* ctx, jp_cost_model* model) {
    if (!ctx || !model) return JP_EINVAL;
    *model = ctx->cost;
    return JP_OK;
}

int jp_set_gemm_tile(jp_ctx* ctx, int width, int64_t auto_max_tiles) {
    if (!ctx) return JP_EINVAL;
    if (width != 0 && width != 128 && width != 256) return fail(ctx, JP_EINVAL, "tile width must be 0, 128 or 256");
    if (auto_max_tiles < 0) return fail(ctx, JP_EINVAL, "auto_max_tiles must be >= 0");
    ctx->gemm_width = width;
    ctx->gemm_auto_tiles = auto_max_tiles;
    return JP_OK;
}

int jp_get_gemm_tile(const jp_ctx* ctx, int* width, int64_t* auto_max_tiles) {
    if (!ctx || !width || !auto_max_tiles) return JP_EINVAL;
    *width = ctx->gemm_width;
    *auto_max_tiles = ctx->gemm_auto_tiles;
    return JP_OK;
}

int jp_set_stream(jp_ctx* ctx, void* stream) {
    if (!ctx) return JP_EINVAL;
    ctx->stream = (cudaStream_t)stream;
    ctx->ws.stream = ctx->stream;
    return JP_OK;
}

int jp_two_path(jp_ctx* ctx, const jp_rel* R, const jp_rel* S, jp_result* out) {
    return run_two_path(ctx, R, S, out, nullptr);
}

int jp_two_path_into(jp_ctx* ctx, const jp_rel* R, const jp_rel* S, int32_t* out_x, int32_t* out_z,
                     int64_t cap, int64_t* count) {
    if (!ctx) return JP_EINVAL;
    if (!count) return fail(ctx, JP_EINVAL, "count is NULL");
    *count = 0;
    if (cap < 0 || (cap > 0 && (!out_x || !out_z))) return fail(ctx, JP_EINVAL, "bad output buffers");
    jp_result res;
    const ExtOut ext{out_x, out_z, cap, count};
    const int rc = run_two_path(ctx, R, S, &res, nullptr, nullptr, &ext);
    if (rc != JP_OK && !(rc == JP_EOVERFLOW && *count > cap)) *count = 0;
    return rc;
}

int jp_two_path_batch(jp_ctx* ctx, const jp_rel* all, int32_t nq, const int64_t* qoff,
                      jp_result* out, int64_t* out_off) {
    if (!ctx) return JP_EINVAL;
    if (!out) return fail(ctx, JP_EINVAL, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    out->k = 2;
    if (!all || !qoff || !out_off) return fail(ctx, JP_EINVAL, "NULL argument");
    if (nq < 1) return fail(ctx, JP_EINVAL, "a batch needs at least one query");
    if (qoff[0] != 0 || qoff[nq] != all->n)
        return fail(ctx, JP_EINVAL, "query offsets must start at 0 and end at the tuple count");
    for (int32_t q = 0; q < nq; ++q)
        if (qoff[q + 1] < qoff[q]) return fail(ctx, JP_EINVAL, "query offsets must not decrease");
    const BatchArgs b{nq, qoff, out_off};
    return run_two_path(ctx, all, nullptr, out, &b);
}

int jp_two_path_filter(jp_ctx* ctx, const jp_rel* R, const jp_rel* S, const jp_rel* T,
                       jp_result* out) {
    if (!ctx) return JP_EINVAL;
    if (!T) return fail(ctx, JP_EINVAL, "T is NULL");
    return run_two_path(ctx, R, S, out, nullptr, T);
}

int jp_set_count_chunk(jp_ctx* ctx, int64_t candidates) {
    if (!ctx) return JP_EINVAL;
    if (candidates < 1) return fail(ctx, JP_EINVAL, "candidates must be >= 1");
    ctx->count_chunk = candidates;
    return JP_OK;
}

int jp_two_path_counts(jp_ctx* ctx, const jp_rel* R, const jp_rel* S, int64_t c_min, int order,
                       jp_result* out) {
    if (!ctx) return JP_EINVAL;
    if (!out) return fail(ctx, JP_EINVAL, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    out->k = 3;
    if (c_min < 1) return fail(ctx, JP_EINVAL, "c_min must be >= 1");
    if (order != JP_ORDER_PAIRS && order != JP_ORDER_COUNT) return fail(ctx, JP_EINVAL, "unknown order");
    int rc = check_rel(ctx, R, "R");
    if (rc) return rc;
    if (S && (rc = check_rel(ctx, S, "S"))) return rc;
    if (S && R->n + S->n >= ((int64_t)1 << 31)) return fail(ctx, JP_EUNSUPPORTED, "R and S together hold 2^31 or more tuples");
    const auto t_start = std::chrono::steady_clock::now();
    void* block = nullptr;
    size_t block_bytes = 0;
    try {
        JP_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = ctx->stream;
        ctx->ws.begin();
        const int64_t launches0 = jp::g_launches;
        JP_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), st));
        for (int i = 0; i < jp::TM_SLOTS; ++i) ctx->tm.used[i] = false;
        ctx->tm.st = st;
        jp::g_timer = &ctx->tm;
        ctx->tm.begin(jp::TM_TOTAL);
        const jp_rel Rd = to_device(ctx, R);
        jp_rel Sd;
        if (S) Sd = to_device(ctx, S);
        const bool self = (S == nullptr) || (S->x == R->x && S->y == R->y && S->n == R->n);
        jp::Graph g;
        ctx->tm.begin(jp::TM_BUILD);
        jp::build_graph(&Rd, self ? nullptr : &Sd, g, ctx->ws, st, ctx->d_status, ctx->hist_host,
                        ctx->host_scalars);
        ctx->tm.end(jp::TM_BUILD);
        jp::Partition p;
        double out_est = 0;
        int judged = 0;
        ctx->tm.begin(jp::TM_SELECT);
        jp::select_thresholds(g, ctx->mode, ctx->d1, ctx->d2, &p.d1, &p.d2, &out_est, ctx->ws, st,
                              ctx->cost, ctx->predictor, &judged);
        ctx->tm.end(jp::TM_SELECT);
        ctx->tm.begin(jp::TM_PARTITION);
        jp::build_partition(g, p, ctx->ws, st, ctx->host_scalars);
        ctx->tm.end(jp::TM_PARTITION);
        jp::Heavy h;
        ctx->tm.begin(jp::TM_PACK);
        jp::heavy_pack(g, p, h, ctx->ws, st);
        ctx->tm.end(jp::TM_PACK);
        jp::CountResult cr;
        jp::count_pairs(g, p, h, c_min, order, cr, ctx->ws, st, ctx->d_status, ctx->hist_host,
                        ctx->count_chunk);
        status_check(ctx);
        if (cr.n > 0) {
            const size_t col = ((size_t)cr.n * sizeof(int32_t) + 255) & ~(size_t)255;
            block_bytes = 3 * col + 256;
            block = ctx->ws.raw_alloc(block_bytes);
            if (!block) throw jp::Error{JP_ENOMEM, "result allocation failed"};
            const int32_t* src[3] = {cr.x, cr.z, cr.cnt};
            for (int i = 0; i < 3; ++i) {
                out->col[i] = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(block) + i * col);
                JP_CUDA_TRY(cudaMemcpyAsync(out->col[i], src[i], (size_t)cr.n * sizeof(int32_t),
                                            cudaMemcpyDeviceToDevice, st));
            }
        }
        ctx->tm.end(jp::TM_TOTAL);
        status_check(ctx);
        jp::g_timer = nullptr;
        out->count = cr.n;
        out->_block = block;
        out->_bytes = block_bytes;
        jp_stats& s = ctx->stats;
        std::memset(&s, 0, sizeof(s));
        s.n_r = g.nr;
        s.n_s = g.ns;
        s.dom_x = g.nx;
        s.dom_y = g.ny;
        s.dom_z = g.nz;
        s.out_join = g.out_join;
        s.out_estimate = out_est;
        s.delta1 = p.d1;
        s.delta2 = p.d2;
        s.threshold_mode = ctx->mode;
        s.u = p.u;
        s.v = p.v;
        s.w = p.w;
        s.light_candidates = cr.candidates;
        s.out_count = cr.n;
        s.learned_judged = judged;
        s.kernel_launches = jp::g_launches - launches0;
        s.gemm_tile = h.present ? h.tbn : 0;
        for (int i = 0; i < jp::TM_SLOTS; ++i) s.ms_pass[i] = ctx->tm.ms(i);
        s.ms_pass[13] = cr.ms_fill;
        s.ms_pass[14] = cr.ms_sort;
        s.ms_pass[15] = cr.ms_merge;
        s.count_ranges = cr.ranges;
        s.count_light_pairs = cr.light_pairs;
        s.heavy_pairs = cr.heavy_pairs;
        s.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        ctx->have_stats = true;
        ctx->err.clear();
        return JP_OK;
    } catch (const jp::Error& e) {
        jp::g_timer = nullptr;
        if (block) ctx->ws.raw_free(block, block_bytes);
        std::memset(out, 0, sizeof(*out));
        return fail(ctx, e.code, e.msg);
    } catch (const std::bad_alloc&) {
        jp::g_timer = nullptr;
        if (block) ctx->ws.raw_free(block, block_bytes);
        std::memset(out, 0, sizeof(*out));
        return fail(ctx, JP_ENOMEM, "host allocation failed");
    }
}

int jp_measure_peaks(jp_ctx* ctx, double* fp8_tflops, double* int8_mma_sync_tflops) {
    if (!ctx || !fp8_tflops || !int8_mma_sync_tflops) return ctx ? fail(ctx, JP_EINVAL, "NULL argument") : JP_EINVAL;
    try {
        JP_CUDA_TRY(cudaSetDevice(ctx->device));
        int sms = 0;
        JP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
        ctx->ws.begin();
        JP_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), ctx->stream));
        jp::measure_peaks(sms, fp8_tflops, int8_mma_sync_tflops, ctx->d_status, ctx->ws, ctx->stream);
        status_check(ctx);
    } catch (const jp::Error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return JP_OK;
}

int jp_selftest_wait(jp_ctx* ctx, int64_t wait_ns) {
    if (!ctx) return JP_EINVAL;
    if (wait_ns < 1 || wait_ns > 5000000000LL) return fail(ctx, JP_EINVAL, "wait_ns out of range");
    try {
        JP_CUDA_TRY(cudaSetDevice(ctx->device));
        JP_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), ctx->stream));
        jp::wait_selftest(ctx->d_status, wait_ns, ctx->stream);
        status_check(ctx);
    } catch (const jp::Error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return fail(ctx, JP_ECUDA, "the self-test wait did not run out");
}

int jp_star(jp_ctx* ctx, int k, const jp_rel* rels, jp_result* out) {
    if (!ctx) return JP_EINVAL;
    if (!out) return fail(ctx, JP_EINVAL, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    if (k < 2 || k > 8) return fail(ctx, JP_EINVAL, "k must be in [2, 8]");
    if (!rels) return fail(ctx, JP_EINVAL, "rels is NULL");
    for (int i = 0; i < k; ++i) {
        int rc = check_rel(ctx, &rels[i], "rels[i]");
        if (rc) return rc;
    }
    if (k == 2) {  // Q*_2 is the two-path query with S = R2
        int rc = jp_two_path(ctx, &rels[0], &rels[1], out);
        out->k = 2;
        return rc;
    }
    const auto t_start = std::chrono::steady_clock::now();
    void* block = nullptr;
    size_t block_bytes = 0;
    out->k = k;
    try {
        JP_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = ctx->stream;
        ctx->ws.begin();
        const int64_t launches0 = jp::g_launches;
        JP_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), st));
        for (int i = 0; i < jp::TM_SLOTS; ++i) ctx->tm.used[i] = false;
        ctx->tm.st = st;
        jp::g_timer = &ctx->tm;
        ctx->tm.begin(jp::TM_TOTAL);
        jp_rel rd[8];
        for (int i = 0; i < k; ++i) rd[i] = to_device(ctx, &rels[i]);

        ctx->tm.begin(jp::TM_BUILD);
        // k > 3: R3..Rk grouped on y from the right into one relation whose x
        // is a group id; Q*_k is Q*_3 over (R1, R2, that relation), its third
        // column expanded back through the groups' value tables
        jp::PairRel levels[6];
        jp::StarChain chain;
        if (k > 3) {
            jp_rel tail = rd[k - 1];
            for (int i = k - 2; i >= 2; --i) {
                jp::pair_relation(&rd[i], &tail, levels[i - 2], ctx->ws, st, ctx->hist_host);
                tail = jp_rel{levels[i - 2].x, levels[i - 2].y, levels[i - 2].n};
            }
            rd[2] = tail;
            chain.levels = k - 3;
            for (int l = 0; l < k - 3; ++l) {
                chain.gp[l] = levels[l].gp;
                chain.gq[l] = levels[l].gq;
            }
        }
        jp::StarOut so;
        jp::run_star3(rd, ctx->mode, ctx->d1, ctx->d2, so, ctx->ws, st, ctx->d_status,
                      ctx->hist_host);
        ctx->tm.end(jp::TM_BUILD);
        jp::Heavy h;
        ctx->tm.begin(jp::TM_PACK);
        jp::heavy_pack(so.g, so.p, h, ctx->ws, st);
        h.tbn = jp::pick_tile(h, ctx->gemm_width, ctx->gemm_auto_tiles);
        ctx->tm.end(jp::TM_PACK);
        jp::heavy_gemm(h, so.p, ctx->d_status, st, nullptr);
        jp::LightResult lr;
        jp::light_and_union(so.g, so.p, h, lr, ctx->ws, st, ctx->d_status, ctx->host_scalars);
        int64_t* out_off = ctx->ws.get<int64_t>(so.g.nx + 1);
        ctx->tm.begin(jp::TM_COUNT);
        const int64_t count = jp::output_count(so.g, lr, out_off, ctx->ws, st, ctx->host_scalars);
        ctx->tm.end(jp::TM_COUNT);
        status_check(ctx);
        if (count > 0) {
            const size_t col_bytes = ((size_t)count * sizeof(int32_t) + 255) & ~(size_t)255;
            block_bytes = (size_t)k * col_bytes;
            block = ctx->ws.raw_alloc(block_bytes);
            if (!block) throw jp::Error{JP_ENOMEM, "result allocation failed"};
            for (int i = 0; i < k; ++i)
                out->col[i] = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(block) + i * col_bytes);
            ctx->tm.begin(jp::TM_PLACE);
            jp::output_write_rows(so.g, lr, out_off, count, so.row1, so.row2, out->col[0],
                                  out->col[1], out->col[2], st);
            if (k > 3) {   // column 2 holds group ids: expand them in place into columns 2..k-1
                int32_t** cols = ctx->ws.get<int32_t*>(8);
                JP_CUDA_TRY(cudaMemcpyAsync(cols, out->col + 2, (size_t)(k - 2) * sizeof(int32_t*),
                                            cudaMemcpyHostToDevice, st));
                jp::star_expand(out->col[2], count, chain, cols, st);
            }
            ctx->tm.end(jp::TM_PLACE);
        }
        ctx->tm.end(jp::TM_TOTAL);
        status_check(ctx);
        jp::g_timer = nullptr;
        out->count = count;
        out->_block = block;
        out->_bytes = block_bytes;

        jp_stats& s = ctx->stats;
        std::memset(&s, 0, sizeof(s));
        s.n_r = so.n_rel[0];
        s.n_s = so.n_rel[1];
        s.dom_x = so.nx[0];
        s.dom_y = so.ny;
        s.dom_z = so.nx[2];
        s.out_join = so.out_join;
        s.out_estimate = so.out_join;
        s.delta1 = so.d1;
        s.delta2 = so.d2;
        s.threshold_mode = ctx->mode;
        s.u = so.p.u;
        s.v = so.p.v;
        s.w = so.p.w;
        s.light_candidates = lr.candidates;
        s.out_count = count;
        s.kernel_launches = jp::g_launches - launches0;
        s.gemm_tile = h.present ? h.tbn : 0;
        for (int q = 0; q < 8; ++q) {
            s.light_x[q] = lr.class_x[q];
            s.light_cand[q] = lr.class_cand[q];
            s.light_deg[q] = lr.class_deg[q];
        }
        for (int i = 0; i < jp::TM_SLOTS; ++i) s.ms_pass[i] = ctx->tm.ms(i);
        s.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        ctx->have_stats = true;
        ctx->err.clear();
        return JP_OK;
    } catch (const jp::Error& e) {
        jp::g_timer = nullptr;
        if (block) ctx->ws.raw_free(block, block_bytes);
        std::memset(out, 0, sizeof(*out));
        return fail(ctx, e.code, e.msg);
    } catch (const std::bad_alloc&) {
        jp::g_timer = nullptr;
        if (block) ctx->ws.raw_free(block, block_bytes);
        std::memset(out, 0, sizeof(*out));
        return fail(ctx, JP_ENOMEM, "host allocation failed");
    }
}

int jp_star_batch(jp_ctx* ctx, int32_t nq, const jp_rel* rels, const int64_t* qoff, jp_result* out,
                  int64_t* out_off) {
    if (!ctx) return JP_EINVAL;
    if (!out) return fail(ctx, JP_EINVAL, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    out->k = 3;
    if (!rels || !qoff || !out_off) return fail(ctx, JP_EINVAL, "NULL argument");
    if (nq < 1) return fail(ctx, JP_EINVAL, "a batch needs at least one query");
    for (int i = 0; i < 3; ++i) {
        int rc = check_rel(ctx, &rels[i], "rels[i]");
        if (rc) return rc;
        const int64_t* qo = qoff + (size_t)i * (nq + 1);
        if (qo[0] != 0 || qo[nq] != rels[i].n)
            return fail(ctx, JP_EINVAL, "query offsets must start at 0 and end at the tuple count");
        for (int32_t q = 0; q < nq; ++q)
            if (qo[q + 1] < qo[q]) return fail(ctx, JP_EINVAL, "query offsets must not decrease");
    }
    if (rels[0].n + rels[1].n + rels[2].n >= ((int64_t)1 << 31))
        return fail(ctx, JP_EUNSUPPORTED, "the relations together hold 2^31 or more tuples");
    if (rels[0].n == 0 || rels[1].n == 0 || rels[2].n == 0) {   // no query has a triple
        for (int32_t q = 0; q <= nq; ++q) out_off[q] = 0;
        std::memset(&ctx->stats, 0, sizeof(ctx->stats));
        ctx->have_stats = true;
        return JP_OK;
    }
    const auto t_start = std::chrono::steady_clock::now();
    void* block = nullptr;
    size_t block_bytes = 0;
    try {
        JP_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = ctx->stream;
        ctx->ws.begin();
        const int64_t launches0 = jp::g_launches;
        JP_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), st));
        for (int i = 0; i < jp::TM_SLOTS; ++i) ctx->tm.used[i] = false;
        ctx->tm.st = st;
        jp::g_timer = &ctx->tm;
        ctx->tm.begin(jp::TM_TOTAL);
        jp_rel rd[3];
        for (int i = 0; i < 3; ++i) rd[i] = to_device(ctx, &rels[i]);
        ctx->tm.begin(jp::TM_BUILD);
        jp::StarBatchIds sb;
        jp::star_batch_encode(rd, nq, qoff, sb, ctx->ws, st, ctx->hist_host, ctx->d_status);
        jp::StarOut so;
        jp::run_star3(sb.rel, ctx->mode, ctx->d1, ctx->d2, so, ctx->ws, st, ctx->d_status,
                      ctx->hist_host);
        ctx->tm.end(jp::TM_BUILD);
        jp::Heavy h;
        ctx->tm.begin(jp::TM_PACK);
        jp::heavy_pack(so.g, so.p, h, ctx->ws, st);
        h.tbn = jp::pick_tile(h, ctx->gemm_width, ctx->gemm_auto_tiles);
        ctx->tm.end(jp::TM_PACK);
        jp::heavy_gemm(h, so.p, ctx->d_status, st, nullptr);
        jp::LightResult lr;
        jp::light_and_union(so.g, so.p, h, lr, ctx->ws, st, ctx->d_status, ctx->host_scalars);
        int64_t* oo = ctx->ws.get<int64_t>(so.g.nx + 1);
        ctx->tm.begin(jp::TM_COUNT);
        const int64_t count = jp::output_count(so.g, lr, oo, ctx->ws, st, ctx->host_scalars);
        ctx->tm.end(jp::TM_COUNT);
        status_check(ctx);
        int32_t* cols[3] = {nullptr, nullptr, nullptr};
        if (count > 0) {
            const size_t col_bytes = ((size_t)count * sizeof(int32_t) + 255) & ~(size_t)255;
            block_bytes = 3 * col_bytes;
            block = ctx->ws.raw_alloc(block_bytes);
            if (!block) throw jp::Error{JP_ENOMEM, "result allocation failed"};
            for (int i = 0; i < 3; ++i)
                cols[i] = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(block) + i * col_bytes);
            ctx->tm.begin(jp::TM_PLACE);
            jp::output_write_rows(so.g, lr, oo, count, so.row1, so.row2, cols[0], cols[1], cols[2],
                                  st);
            ctx->tm.end(jp::TM_PLACE);
        }
        jp::star_batch_finish(cols, count, sb, nq, out_off, ctx->ws, st);
        ctx->tm.end(jp::TM_TOTAL);
        status_check(ctx);
        jp::g_timer = nullptr;
        for (int i = 0; i < 3; ++i) out->col[i] = cols[i];
        out->count = count;
        out->_block = block;
        out->_bytes = block_bytes;
        jp_stats& s = ctx->stats;
        std::memset(&s, 0, sizeof(s));
        s.n_r = so.n_rel[0];
        s.n_s = so.n_rel[1];
        s.dom_x = so.nx[0];
        s.dom_y = so.ny;
        s.dom_z = so.nx[2];
        s.out_join = so.out_join;
        s.out_estimate = so.out_join;
        s.delta1 = so.d1;
        s.delta2 = so.d2;
        s.threshold_mode = ctx->mode;
        s.u = so.p.u;
        s.v = so.p.v;
        s.w = so.p.w;
        s.light_candidates = lr.candidates;
        s.out_count = count;
        s.kernel_launches = jp::g_launches - launches0;
        s.gemm_tile = h.present ? h.tbn : 0;
        for (int i = 0; i < jp::TM_SLOTS; ++i) s.ms_pass[i] = ctx->tm.ms(i);
        s.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        ctx->have_stats = true;
        ctx->err.clear();
        return JP_OK;
    } catch (const jp::Error& e) {
        jp::g_timer = nullptr;
        if (block) ctx->ws.raw_free(block, block_bytes);
        std::memset(out, 0, sizeof(*out));
        return fail(ctx, e.code, e.msg);
    } catch (const std::bad_alloc&) {
        jp::g_timer = nullptr;
        if (block) ctx->ws.raw_free(block, block_bytes);
        std::memset(out, 0, sizeof(*out));
        return fail(ctx, JP_ENOMEM, "host allocation failed");
    }
}

int jp_set_predictor(jp_ctx* ctx, jp_mlp* model) {
    if (!ctx) return JP_EINVAL;
    ctx->predictor = model;
    return JP_OK;
}

int jp_features(jp_ctx* ctx, const jp_rel* R, const jp_rel* S, float* out128) {
    if (!ctx) return JP_EINVAL;
    if (!out128) return fail(ctx, JP_EINVAL, "out128 is NULL");
    int rc = check_rel(ctx, R, "R");
    if (rc) return rc;
    if (S && (rc = check_rel(ctx, S, "S"))) return rc;
    try {
        JP_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = ctx->stream;
        ctx->ws.begin();
        JP_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), st));
        jp_rel Rd = to_device(ctx, R);
        jp_rel Sd;
        if (S) Sd = to_device(ctx, S);
        const bool self = (S == nullptr) || (S->x == R->x && S->y == R->y && S->n == R->n);
        jp::Graph g;
        jp::build_graph(&Rd, self ? nullptr : &Sd, g, ctx->ws, st, ctx->d_status, ctx->hist_host,
                        ctx->host_scalars);
        jp::graph_features(g, out128, ctx->ws, st);
        status_check(ctx);
    } catch (const jp::Error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return JP_OK;
}

int jp_get_stats(const jp_ctx* ctx, jp_stats* stats) {
    if (!ctx || !stats) return JP_EINVAL;
    *stats = ctx->stats;
    return ctx->have_stats ? JP_OK : JP_EINVAL;
}

int jp_result_to_host(jp_ctx* ctx, const jp_result* res, int32_t* const* host_cols) {
    if (!ctx || !res || (!host_cols && res->count > 0)) return JP_EINVAL;
    try {
        JP_CUDA_TRY(cudaSetDevice(ctx->device));
        for (int i = 0; i < res->k && res->count > 0; ++i) {
            if (!host_cols[i] || !res->col[i]) return fail(ctx, JP_EINVAL, "NULL column");
            JP_CUDA_TRY(cudaMemcpyAsync(host_cols[i], res->col[i], (size_t)res->count * sizeof(int32_t),
                                        cudaMemcpyDeviceToHost, ctx->stream));
        }
        JP_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    } catch (const jp::Error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return JP_OK;
}

void jp_result_free(jp_ctx* ctx, jp_result* res) {
    if (!ctx || !res) return;
    if (res->_block) ctx->ws.raw_free(res->_block, res->_bytes);
    std::memset(res, 0, sizeof(*res));
}

const char* jp_last_error(const jp_ctx* ctx) {
    if (!ctx) return "NULL context";
    return ctx->err.c_str();
}

}  // extern "C"
