// Output placement (the final union pass of Algorithm 1): every x's sorted
// distinct z list is moved from the scratch buffer to its place in the
// globally sorted result, and ids are mapped back to int32 values.
//
// Because x ids and z ids are assigned in value order, writing the lists in
// x-id order with each list in z-id order gives the lexicographic order of
// the signed values.  The write is load balanced over output positions: each
// thread owns a run of consecutive outputs, finds its x by binary search on
// the output offsets once, and then walks forward.
#include "jp_internal.cuh"

namespace jp {
namespace {

constexpr int OUT_THREADS = 256;
constexpr int OUT_VT = 8;

__global__ void widen_kernel(const int32_t* in, int64_t n, int64_t* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i];
}

__global__ void place_kernel(const int64_t* __restrict__ out_off, int64_t nx,
                             const int64_t* __restrict__ tmp_off, const int32_t* __restrict__ tmp,
                             const int32_t* __restrict__ xval, const int32_t* __restrict__ zval,
                             int64_t count, int32_t* __restrict__ out_x,
                             int32_t* __restrict__ out_z) {
    const int64_t first = ((int64_t)blockIdx.x * OUT_THREADS + threadIdx.x) * OUT_VT;
    if (first >= count) return;
    // largest x with out_off[x] <= first
    int64_t lo = 0, hi = nx;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (out_off[mid] <= first) lo = mid; else hi = mid;
    }
    int64_t x = lo;
    int64_t next = (x + 1 < nx) ? out_off[x + 1] : count;
#pragma unroll
    for (int i = 0; i < OUT_VT; ++i) {
        const int64_t o = first + i;
        if (o >= count) break;
        while (o >= next) {
            ++x;
            next = (x + 1 < nx) ? out_off[x + 1] : count;
        }
        const int32_t z = tmp[tmp_off[x] + (o - out_off[x])];
        out_x[o] = xval[x];
        out_z[o] = zval[z];
    }
}

}  // namespace

int64_t output_count(const Graph& g, const LightResult& lr, int64_t* out_off, Arena& ws,
                     cudaStream_t st, int64_t* host_scalars) {
    (void)host_scalars;
    const int64_t nx = g.nx;
    int64_t* wide = ws.get<int64_t>(nx + 1);
    int64_t* d_total = ws.get<int64_t>(1);
    if (nx > 0) {
        widen_kernel<<<grid_for(nx, 256, 152 * 16), 256, 0, st>>>(lr.cnt, nx, wide);
        JP_CHECK_LAUNCH();
    }
    scan_i64(wide, out_off, nx, d_total, ws, st);
    int64_t total = 0;
    JP_CUDA_TRY(cudaMemcpyAsync(&total, d_total, sizeof(total), cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaStreamSynchronize(st));
    return total;
}

void output_write(const Graph& g, const LightResult& lr, const int64_t* out_off, int64_t count,
                  int32_t* out_x, int32_t* out_z, cudaStream_t st) {
    if (count <= 0) return;
    const int64_t per_block = (int64_t)OUT_THREADS * OUT_VT;
    const int64_t blocks = (count + per_block - 1) / per_block;
    place_kernel<<<(unsigned)blocks, OUT_THREADS, 0, st>>>(out_off, g.nx, lr.tmp_off, lr.tmp,
                                                          g.xval, g.zval, count, out_x, out_z);
    JP_CHECK_LAUNCH();
}

}  // namespace jp
