// Output placement (the final union pass of Algorithm 1): every x's sorted
// distinct z list is moved from the scratch buffer to its place in the
// globally sorted result; the lists of bitmap rows hold z ids, which are
// mapped to values here (the other lists already hold values).
//
// Because x ids and z ids are assigned in value order, writing the lists in
// x-id order with each list in z-id order gives the lexicographic order of
// the signed values.  The write is load balanced over output positions: a
// block owns one tile of consecutive outputs, reads the x range of its tile
// from a precomputed tile -> x table, stages that range's offsets in shared
// memory and writes striped, coalesced output.
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

constexpr int OUT_SX = 512;   // x entries staged in shared memory per tile

// largest x in [lo, hi) with off[x] <= o (off non-decreasing, off[lo] <= o)
__device__ __forceinline__ int64_t find_x(const int64_t* off, int64_t lo, int64_t hi, int64_t o) {
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= o) lo = mid; else hi = mid;
    }
    return lo;
}

// Entry i of a row's list (see TMP_IDS): a z value read from tmp or in place
// from szval, or, for bitmap rows, a z id (*is_id set) to be mapped by zval.
__device__ __forceinline__ int32_t list_at(const int32_t* tmp, const int32_t* szval, int64_t toff,
                                           int64_t i, bool* is_id) {
    if (toff < 0) {
        *is_id = false;
        return szval[-toff - 1 + i];
    }
    *is_id = (toff & TMP_IDS) != 0;
    return tmp[(toff & ~TMP_IDS) + i];
}

// tile_x[t] = the x whose output range holds output t * tile (thread per x:
// an x marks every tile that starts inside its range)
__global__ void tile_start_kernel(const int64_t* __restrict__ out_off, int64_t nx, int64_t count,
                                  int64_t tile, int32_t* __restrict__ tile_x) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nx;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = out_off[x];
        const int64_t e = (x + 1 < nx) ? out_off[x + 1] : count;
        for (int64_t t = (b + tile - 1) / tile; t * tile < e; ++t) tile_x[t] = (int32_t)x;
    }
}

// One tile of OUT_THREADS * OUT_VT consecutive outputs per block; when the
// tile's x range is short its offsets are staged in shared memory.  Thread t
// writes outputs o0 + t + k*OUT_THREADS, so each store instruction of a warp
// covers 32 consecutive outputs.
// X2: a second row column (the star's x2) is written next to the first.
// VMAP: x and z values are ids into vmap, which gives the written values.
// Bound by latency: a thread's loads are the only work in flight, so the
// launch bound asks for 6 resident blocks per SM (1,536 threads, at most 40
// registers each).  With the row walk, 8 blocks per SM (32 registers) spill
// and measured slower; without it 8 was the best.
template <bool X2, bool VMAP>
__global__ void __launch_bounds__(OUT_THREADS, 6)
    place_kernel(const int64_t* __restrict__ out_off, int64_t nx,
                             const int32_t* __restrict__ tile_x,
                             const int64_t* __restrict__ tmp_off, const int32_t* __restrict__ tmp,
                             const int32_t* __restrict__ szval,
                             const int32_t* __restrict__ xval, const int32_t* __restrict__ xval2,
                             const int32_t* __restrict__ zval, int64_t count,
                             int32_t* __restrict__ out_x, int32_t* __restrict__ out_x2,
                             int32_t* __restrict__ out_z, const int32_t* __restrict__ vmap) {
    __shared__ int64_t s_off[OUT_SX + 1];
    __shared__ int64_t s_toff[OUT_SX];
    __shared__ int32_t s_xv[OUT_SX];
    __shared__ int32_t s_xv2[OUT_SX];
    const int64_t o0 = (int64_t)blockIdx.x * OUT_THREADS * OUT_VT;
    const int64_t o_last = min(count, o0 + (int64_t)OUT_THREADS * OUT_VT) - 1;
    // x range of the tile: from the x holding its first output to the x holding
    // the next tile's first output (an upper bound of the x holding o_last)
    const int64_t xlo = tile_x[blockIdx.x];
    const int64_t xhi = (o_last + 1 < count) ? (int64_t)tile_x[blockIdx.x + 1] + 1 : nx;
    const int64_t nxs = xhi - xlo;
    const bool staged = nxs <= OUT_SX;
    if (staged) {
        for (int64_t i = threadIdx.x; i < nxs; i += OUT_THREADS) {
            s_off[i] = out_off[xlo + i];
            s_toff[i] = tmp_off[xlo + i];
            s_xv[i] = VMAP ? vmap[xval[xlo + i]] : xval[xlo + i];
            if (X2) s_xv2[i] = xval2[xlo + i];
        }
        if (threadIdx.x == 0) s_off[nxs] = (xhi < nx) ? out_off[xhi] : count;
    }
    __syncthreads();
    // all of a thread's list reads, then all of its id -> value gathers, then
    // the stores: OUT_VT independent loads in flight per phase
    int32_t zv[OUT_VT], xv[OUT_VT], xv2[OUT_VT];
    uint32_t ids = 0;   // bit k: zv[k] is a z id
    int64_t ri = -1, r_beg = 0, r_end = -1, r_toff = 0;   // the current staged row
    int32_t r_xv = 0, r_xv2 = 0;
#pragma unroll
    for (int k = 0; k < OUT_VT; ++k) {
        const int64_t o = o0 + threadIdx.x + (int64_t)k * OUT_THREADS;
        zv[k] = 0;
        xv[k] = 0;
        xv2[k] = 0;
        bool is_id = false;
        if (o <= o_last) {
            if (staged) {
                // a thread's outputs (OUT_THREADS apart) only move forward through
                // the rows: it keeps its current row's bounds and values in
                // registers and reads shared memory again only past the row's end
                if (o >= r_end) {
                    // the next row when it holds o, else a search past the current one
                    const int64_t i = (ri >= 0 && ri + 2 <= nxs && o < s_off[ri + 2])
                                          ? ri + 1
                                          : find_x(s_off, ri < 0 ? 0 : ri + 1, nxs, o);
                    ri = i;
                    r_beg = s_off[i];
                    r_end = s_off[i + 1];
                    r_toff = s_toff[i];
                    r_xv = s_xv[i];
                    if (X2) r_xv2 = s_xv2[i];
                }
                zv[k] = list_at(tmp, szval, r_toff, o - r_beg, &is_id);
                xv[k] = r_xv;
                if (X2) xv2[k] = r_xv2;
            } else {
                const int64_t x = find_x(out_off, xlo, xhi, o);
                zv[k] = list_at(tmp, szval, tmp_off[x], o - out_off[x], &is_id);
                xv[k] = VMAP ? vmap[xval[x]] : xval[x];
                if (X2) xv2[k] = xval2[x];
            }
        }
        ids |= (uint32_t)is_id << k;
    }
#pragma unroll
    for (int k = 0; k < OUT_VT; ++k)
        if (ids >> k & 1u) zv[k] = zval[zv[k]];
    if (VMAP) {
#pragma unroll
        for (int k = 0; k < OUT_VT; ++k)
            if (o0 + threadIdx.x + (int64_t)k * OUT_THREADS <= o_last) zv[k] = vmap[zv[k]];
    }
#pragma unroll
    for (int k = 0; k < OUT_VT; ++k) {
        const int64_t o = o0 + threadIdx.x + (int64_t)k * OUT_THREADS;
        if (o <= o_last) {
            out_x[o] = xv[k];
            if (X2) out_x2[o] = xv2[k];
            out_z[o] = zv[k];
        }
    }
}

}  // namespace

int64_t output_count(const Graph& g, LightResult& lr, int64_t* out_off, Arena& ws,
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
    const int64_t tile = (int64_t)OUT_THREADS * OUT_VT;
    const int64_t ntiles = (total + tile - 1) / tile;
    lr.tile_x = ws.get<int32_t>(ntiles + 1);
    if (total > 0) {
        tile_start_kernel<<<grid_for(nx, 256, 152 * 16), 256, 0, st>>>(out_off, nx, total, tile,
                                                                       lr.tile_x);
        JP_CHECK_LAUNCH();
    }
    return total;
}

void output_write(const Graph& g, const LightResult& lr, const int64_t* out_off, int64_t count,
                  int32_t* out_x, int32_t* out_z, cudaStream_t st) {
    output_write_rows(g, lr, out_off, count, g.xval, nullptr, out_x, nullptr, out_z, st);
}

void output_write_rows(const Graph& g, const LightResult& lr, const int64_t* out_off,
                       int64_t count, const int32_t* rowval, const int32_t* rowval2,
                       int32_t* out_row, int32_t* out_row2, int32_t* out_z, cudaStream_t st) {
    if (count <= 0) return;
    const int64_t per_block = (int64_t)OUT_THREADS * OUT_VT;
    const int64_t blocks = (count + per_block - 1) / per_block;
    if (rowval2 && out_row2)
        place_kernel<true, false><<<(unsigned)blocks, OUT_THREADS, 0, st>>>(
            out_off, g.nx, lr.tile_x, lr.tmp_off, lr.tmp, lr.szval, rowval, rowval2, g.zval, count,
            out_row, out_row2, out_z, nullptr);
    else
        place_kernel<false, false><<<(unsigned)blocks, OUT_THREADS, 0, st>>>(
            out_off, g.nx, lr.tile_x, lr.tmp_off, lr.tmp, lr.szval, rowval, nullptr, g.zval, count,
            out_row, nullptr, out_z, nullptr);
    JP_CHECK_LAUNCH();
}

void output_write_mapped(const Graph& g, const LightResult& lr, const int64_t* out_off,
                         int64_t count, const int32_t* vmap, int32_t* out_x, int32_t* out_z,
                         cudaStream_t st) {
    if (count <= 0) return;
    const int64_t per_block = (int64_t)OUT_THREADS * OUT_VT;
    const int64_t blocks = (count + per_block - 1) / per_block;
    place_kernel<false, true><<<(unsigned)blocks, OUT_THREADS, 0, st>>>(
        out_off, g.nx, lr.tile_x, lr.tmp_off, lr.tmp, lr.szval, g.xval, nullptr, g.zval, count,
        out_x, nullptr, out_z, vmap);
    JP_CHECK_LAUNCH();
}

}  // namespace jp
