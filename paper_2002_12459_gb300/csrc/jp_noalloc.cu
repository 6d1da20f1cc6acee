// jp_two_path_noalloc: the two-path query for callers that cannot allocate
// device memory.  It has no counterpart in the paper.
//
// Some callers of this library cannot call cudaMalloc or any other
// allocating routine when they query:
//  - services that reserve their whole device-memory budget at start-up
//    (a serving process whose memory pool already holds nearly all of the
//    GPU) and forbid later allocations, because one more allocation would
//    fail or fragment that budget;
//  - plug-ins running inside a host program that owns every device
//    allocation and gives its extensions none (a database engine's
//    user-defined functions, for example);
//  - latency-bound loops for which an allocation, which can wait for the
//    device, costs more than the query.
// This entry point runs the same pipeline as jp_two_path, but every scratch
// buffer is carved from one file-scope __device__ array of
// JP_NOALLOC_SCRATCH_BYTES, and the result goes to output buffers the caller
// owns.  It calls no cudaMalloc, cudaFree or other allocating routine.
//
// Limits and sharing rules (also stated in jp.h):
//  - queries whose scratch does not fit in the array fail with
//    JP_EUNSUPPORTED; inputs above JP_NOALLOC_MAX_TUPLES are rejected first;
//  - every call shares the array and it keeps the last call's contents; the
//    pipeline clears what must start at zero itself;
//  - calls that overlap on the GPU (other streams, other threads) race on the
//    array: serialise them.  A call returns only after its own work on the
//    stream has finished, failed calls included;
//  - the first call on a device looks the array's device address up with
//    cudaGetSymbolAddress.
#include <cstring>
#include <mutex>
#include <new>

#include "jp_internal.cuh"

namespace {

// The scratch array.  In host code its name is only a host-side stand-in:
// kernels get the device address obtained with cudaGetSymbolAddress.
static __device__ __align__(256) uint8_t g_noalloc_scratch[JP_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
void* g_scratch_addr[MAX_DEVICES] = {};
uint32_t g_hist_host[2048];          // host side of the radix-sort digit histogram
int64_t g_host_scalars[64];

void* no_alloc(size_t, void*, void*) { return nullptr; }
void no_free(void*, size_t, void*, void*) {}

bool on_device(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int jp_two_path_noalloc(const jp_rel* R, const jp_rel* S, int mode, int64_t delta1,
                                   int64_t delta2, int32_t* out_x, int32_t* out_z,
                                   int64_t out_cap, int64_t* out_count, void* stream) {
    if (!R || !out_count) return JP_EINVAL;
    *out_count = 0;
    if (mode != JP_FIXED && mode != JP_CLOSED_FORM) return JP_EINVAL;
    if (mode == JP_FIXED && (delta1 < 1 || delta2 < 1)) return JP_EINVAL;
    if (out_cap < 0 || (out_cap > 0 && (!out_x || !out_z))) return JP_EINVAL;
    const jp_rel* rels[2] = {R, S};
    for (const jp_rel* r : rels) {
        if (!r) continue;
        if (r->n < 0) return JP_EINVAL;
        if (r->n > JP_NOALLOC_MAX_TUPLES) return JP_EUNSUPPORTED;
        if (r->n > 0 && (!on_device(r->x) || !on_device(r->y))) return JP_EINVAL;
    }
    if (out_cap > 0 && (!on_device(out_x) || !on_device(out_z))) return JP_EINVAL;

    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    try {
        int dev = 0;
        JP_CUDA_TRY(cudaGetDevice(&dev));
        if (dev < 0 || dev >= MAX_DEVICES) return JP_EUNSUPPORTED;
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            JP_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
            g_scratch_addr[dev] = p;
        }
        cudaStream_t st = (cudaStream_t)stream;
        jp::Arena ws;
        ws.alloc = no_alloc;          // growth is impossible: a full array fails the query
        ws.release = no_free;
        ws.stream = st;
        ws.chunks.push_back({reinterpret_cast<char*>(g_scratch_addr[dev]),
                             (size_t)JP_NOALLOC_SCRATCH_BYTES});
        ws.reset();
        uint32_t* d_status = ws.get<uint32_t>(1);
        JP_CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st));

        const bool self = (S == nullptr) || (S->x == R->x && S->y == R->y && S->n == R->n);
        jp::Graph g;
        jp::build_graph(R, self ? nullptr : S, g, ws, st, d_status, g_hist_host, g_host_scalars);
        jp::Partition p;
        double out_est = 0;
        jp::select_thresholds(g, mode, delta1, delta2, &p.d1, &p.d2, &out_est, ws, st,
                              jp::default_cost_model());
        jp::build_partition(g, p, ws, st, g_host_scalars);
        jp::Heavy h;
        jp::heavy_pack(g, p, h, ws, st);
        jp::heavy_gemm(h, p, d_status, st, nullptr);
        jp::LightResult lr;
        jp::light_and_union(g, p, h, lr, ws, st, d_status, g_host_scalars);
        int64_t* out_off = ws.get<int64_t>(g.nx + 1);
        const int64_t count = jp::output_count(g, lr, out_off, ws, st, g_host_scalars);
        uint32_t s = 0;
        JP_CUDA_TRY(cudaMemcpyAsync(&s, d_status, sizeof(s), cudaMemcpyDeviceToHost, st));
        JP_CUDA_TRY(cudaStreamSynchronize(st));
        if (s & jp::ST_TIMEOUT) return JP_ETIMEOUT;
        if (s) return JP_EOVERFLOW;
        *out_count = count;
        if (count > out_cap) return JP_EOVERFLOW;   // *out_count tells the size needed
        jp::output_write(g, lr, out_off, count, out_x, out_z, st);
        JP_CUDA_TRY(cudaMemcpyAsync(&s, d_status, sizeof(s), cudaMemcpyDeviceToHost, st));
        JP_CUDA_TRY(cudaStreamSynchronize(st));
        if (s) return JP_EOVERFLOW;
        return JP_OK;
    } catch (const jp::Error& e) {
        // kernels of this call may still be queued: wait for them, so that the
        // next call (on any stream) finds the array idle
        cudaStreamSynchronize((cudaStream_t)stream);
        cudaGetLastError();
        // the only device allocation the pipeline attempts is growing the
        // workspace, which here means the query needs more than the array holds
        return e.code == JP_ENOMEM ? JP_EUNSUPPORTED : e.code;
    } catch (const std::bad_alloc&) {
        cudaStreamSynchronize((cudaStream_t)stream);
        cudaGetLastError();
        return JP_ENOMEM;   // host memory for the pipeline's bookkeeping ran out
    } catch (...) {
        cudaStreamSynchronize((cudaStream_t)stream);
        cudaGetLastError();
        return JP_ECUDA;
    }
}
