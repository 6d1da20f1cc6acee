// Device primitives: exclusive scans, LSD radix sort of 64-bit keys, unique.
//
// These serve the index-building step (Section 5, "Indexing relations": the
// relations are sorted once and indexed both ways) and the offset
// computations of the expansion and output passes.
#include <algorithm>

#include "jp_internal.cuh"

namespace jp {

int grid_for(int64_t n, int block, int max_blocks) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

// ------------------------------------------------------------------ scans
namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ T warp_inclusive(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive scan of one value per thread across the block; *total gets the sum.
template <typename T>
__device__ T block_exclusive(T v, T* sw, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = warp_inclusive(v);
    if (lane == 31) sw[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T s = lane < nw ? sw[lane] : T(0);
        s = warp_inclusive(s);
        if (lane < nw) sw[lane] = s;
    }
    __syncthreads();
    T prefix = warp > 0 ? sw[warp - 1] : T(0);
    *total = sw[nw - 1];
    __syncthreads();
    return prefix + inc - v;
}

template <typename T>
__global__ void scan_reduce_kernel(const T* in, int64_t n, T* partial) {
    __shared__ T sw[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < n) s += in[base + i];
    T tot;
    block_exclusive(s, sw, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <typename T>
__global__ void scan_final_kernel(const T* in, T* out, int64_t n, const T* partial, T* d_total) {
    __shared__ T sw[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = (base + i < n) ? in[base + i] : T(0);
        s += v[i];
    }
    T tot;
    T ex = block_exclusive(s, sw, &tot);
    T off = partial ? partial[blockIdx.x] : T(0);
    T run = off + ex;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (d_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *d_total = off + tot;
}

template <typename T>
void scan_impl(const T* in, T* out, int64_t n, T* d_total, Arena& ws, cudaStream_t st) {
    if (n <= 0) {
        if (d_total) JP_CUDA_TRY(cudaMemsetAsync(d_total, 0, sizeof(T), st));
        return;
    }
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        scan_final_kernel<T><<<1, SCAN_THREADS, 0, st>>>(in, out, n, nullptr, d_total);
        JP_CHECK_LAUNCH();
        return;
    }
    T* partial = ws.get<T>(nb);
    scan_reduce_kernel<T><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, partial);
    JP_CHECK_LAUNCH();
    scan_impl<T>(partial, partial, nb, nullptr, ws, st);
    scan_final_kernel<T><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, out, n, partial, d_total);
    JP_CHECK_LAUNCH();
}

}  // namespace

void scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* d_total, Arena& ws,
              cudaStream_t st) {
    scan_impl<uint32_t>(in, out, n, d_total, ws, st);
}

void scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* d_total, Arena& ws,
              cudaStream_t st) {
    // int64 has no shuffle overload ambiguity issues; use long long arithmetic
    scan_impl<long long>(reinterpret_cast<const long long*>(in), reinterpret_cast<long long*>(out),
                         n, reinterpret_cast<long long*>(d_total), ws, st);
}

// ------------------------------------------------------------- radix sort
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

__global__ void rs_histogram_kernel(const uint64_t* keys, int64_t n, uint32_t* hist) {
    __shared__ uint32_t h[8][256];
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[i];
#pragma unroll
        for (int b = 0; b < 8; ++b) atomicAdd(&h[b][(k >> (8 * b)) & 255], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) {
        uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&hist[i], c);
    }
}

__global__ void rs_upsweep_kernel(const uint64_t* keys, int64_t n, int shift, uint32_t* counts,
                                  int64_t nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int r = 0; r < RS_ITEMS; ++r) {
        int64_t idx = base + (int64_t)r * RS_THREADS + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile of RS_TILE keys.  Warp w owns the keys
// [w * 512, (w + 1) * 512) of the tile and ranks them round by round (32
// consecutive keys a round) with __match_any_sync against a warp-private
// counter per digit; the per-warp counts then give every key its position in
// the tile sorted by digit (warps in order, so the order of equal digits is
// the input order).  The keys are placed there in shared memory and written
// out in that order: runs of one digit go to consecutive addresses.
__global__ void __launch_bounds__(RS_THREADS) rs_downsweep_kernel(const uint64_t* in, uint64_t* out,
                                                                  int64_t n, int shift,
                                                                  const uint32_t* offs, int64_t nblocks) {
    __shared__ uint64_t sk[RS_TILE];
    __shared__ uint32_t cnt[RS_THREADS / 32][256];
    __shared__ uint32_t lstart[256];
    __shared__ uint32_t gbase[256];
    __shared__ uint32_t wsum[RS_THREADS / 32];
    constexpr int WARPS = RS_THREADS / 32;
    constexpr int PER_WARP = RS_TILE / WARPS;   // = 32 * RS_ITEMS
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) cnt[w][t] = 0u;
    gbase[t] = offs[(int64_t)t * nblocks + blockIdx.x];
    __syncthreads();
    const int64_t tb = (int64_t)blockIdx.x * RS_TILE;
    const int64_t wb = tb + (int64_t)warp * PER_WARP;
    const unsigned lt = (1u << lane) - 1u;
    uint64_t k[RS_ITEMS];
    uint32_t rk[RS_ITEMS];
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t idx = wb + r * 32 + lane;
        k[r] = idx < n ? in[idx] : 0ull;
    }
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const bool valid = wb + r * 32 + lane < n;
        const unsigned d = valid ? (unsigned)((k[r] >> shift) & 255) : (256u + lane);
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = valid ? cnt[warp][d] : 0u;
        rk[r] = before + __popc(peers & lt);
        __syncwarp();
        if (valid && (peers & lt) == 0u) cnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // digit t: where each warp's keys of that digit start among the tile's, and the tile's total
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
        const uint32_t c = cnt[w][t];
        cnt[w][t] = tot;
        tot += c;
    }
    // exclusive scan of the totals over the 256 digits
    uint32_t v = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += wsum[w];
    lstart[t] = wpre + v - tot;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        if (wb + r * 32 + lane < n) {
            const unsigned d = (unsigned)((k[r] >> shift) & 255);
            sk[lstart[d] + cnt[warp][d] + rk[r]] = k[r];
        }
    }
    __syncthreads();
    const int tile_n = (int)((n - tb) < RS_TILE ? (n - tb) : RS_TILE);
    for (int i = t; i < tile_n; i += RS_THREADS) {
        const uint64_t key = sk[i];
        const unsigned d = (unsigned)((key >> shift) & 255);
        out[gbase[d] + (uint32_t)(i - (int)lstart[d])] = key;
    }
}

__global__ void unique_mark_kernel(const uint64_t* k, int64_t n, uint32_t* flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || k[i] != k[i - 1]) ? 1u : 0u;
}

__global__ void unique_scatter_kernel(const uint64_t* k, int64_t n, const uint32_t* idx,
                                      uint64_t* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (i == 0 || k[i] != k[i - 1]) out[idx[i]] = k[i];
}

}  // namespace

uint64_t* radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, Arena& ws, cudaStream_t st,
                         uint32_t* hist_host) {
    if (n <= 1) return keys;
    uint32_t* hist = ws.get<uint32_t>(8 * 256);
    JP_CUDA_TRY(cudaMemsetAsync(hist, 0, 8 * 256 * sizeof(uint32_t), st));
    rs_histogram_kernel<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(keys, n, hist);
    JP_CHECK_LAUNCH();
    JP_CUDA_TRY(cudaMemcpyAsync(hist_host, hist, 8 * 256 * sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaStreamSynchronize(st));
    bool need[8];
    for (int b = 0; b < 8; ++b) {
        need[b] = true;
        for (int d = 0; d < 256; ++d)
            if (hist_host[b * 256 + d] == (uint32_t)n) need[b] = false;
    }
    int64_t nb = (n + RS_TILE - 1) / RS_TILE;
    uint32_t* counts = ws.get<uint32_t>(256 * nb);
    uint64_t* src = keys;
    uint64_t* dst = tmp;
    for (int b = 0; b < 8; ++b) {
        if (!need[b]) continue;
        int shift = 8 * b;
        rs_upsweep_kernel<<<(unsigned)nb, RS_THREADS, 0, st>>>(src, n, shift, counts, nb);
        JP_CHECK_LAUNCH();
        scan_u32(counts, counts, 256 * nb, nullptr, ws, st);
        rs_downsweep_kernel<<<(unsigned)nb, RS_THREADS, 0, st>>>(src, dst, n, shift, counts, nb);
        JP_CHECK_LAUNCH();
        std::swap(src, dst);
    }
    return src;
}

void unique_u64(const uint64_t* keys, int64_t n, uint64_t* out, uint32_t* d_count, Arena& ws,
                cudaStream_t st) {
    if (n <= 0) {
        JP_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(uint32_t), st));
        return;
    }
    uint32_t* flag = ws.get<uint32_t>(n);
    uint32_t* idx = ws.get<uint32_t>(n);
    int g = grid_for(n, 256, 152 * 16);
    unique_mark_kernel<<<g, 256, 0, st>>>(keys, n, flag);
    JP_CHECK_LAUNCH();
    scan_u32(flag, idx, n, d_count, ws, st);
    unique_scatter_kernel<<<g, 256, 0, st>>>(keys, n, idx, out);
    JP_CHECK_LAUNCH();
}

}  // namespace jp
