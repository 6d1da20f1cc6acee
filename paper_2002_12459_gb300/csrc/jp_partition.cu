// Heavy/light partition (Section 3.1, Algorithm 1, first two lines).
//
// A value is heavy when its degree exceeds its threshold (light is <=):
//   x heavy  iff deg_R(x) > Delta2          -> rows of M1 (u of them)
//   z heavy  iff deg_S(z) > Delta2          -> columns of M2 (w of them)
//   y heavy  iff max(deg_R(y), deg_S(y)) > Delta1   -> shared inner dimension (v)
// The y rule is the reading that reproduces the Section 3.1 worked example;
// any split gives the same result (the correctness argument after
// Algorithm 1), only the cost changes.  A tuple (a, b) of R is in R^+ iff a
// and b are heavy; (c, b) of S is in S^+ iff c and b are heavy.  Heavy ids
// are assigned in value order.
//
// For the light part of a heavy x the expansion may only take, from a heavy
// y, the light z values (the R^+ join S^- term); those short lists are
// materialised here as a CSR over the heavy y values.
#include "jp_internal.cuh"

namespace jp {
namespace {

inline int G(int64_t n) { return grid_for(n, 256, 152 * 16); }

__global__ void heavy_flag_kernel(const int32_t* deg_a, const int32_t* deg_b, int64_t n,
                                  int64_t thr, uint32_t* flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t d = deg_a[i];
        if (deg_b) d = max(d, deg_b[i]);
        flag[i] = (d > thr) ? 1u : 0u;
    }
}

__global__ void heavy_assign_kernel(const uint32_t* flag, const uint32_t* idx, int64_t n,
                                    int32_t* h, int32_t* h_inv) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (flag[i]) {
            h[i] = (int32_t)idx[i];
            h_inv[idx[i]] = (int32_t)i;
        } else {
            h[i] = -1;
        }
    }
}

// cnt[j] = number of light z in S[b] for heavy y j = hy_inv^-1(b); warp per j
__global__ void light_z_count_kernel(const int32_t* hy_inv, int64_t v, const int32_t* syoff,
                                     const int32_t* szcol, const int32_t* hz, uint32_t* cnt) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = warp; j < v; j += nwarps) {
        int32_t b = hy_inv[j];
        uint32_t c = 0;
        for (int32_t e = syoff[b] + lane; e < syoff[b + 1]; e += 32) c += (hz[szcol[e]] < 0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if (lane == 0) cnt[j] = c;
    }
}

__global__ void light_z_fill_kernel(const int32_t* hy_inv, int64_t v, const int32_t* syoff,
                                    const int32_t* szcol, const int32_t* hz, const uint32_t* off,
                                    int32_t* slcol) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = warp; j < v; j += nwarps) {
        int32_t b = hy_inv[j];
        uint32_t base = off[j];
        int32_t e0 = syoff[b], e1 = syoff[b + 1];
        for (int32_t e = e0; e < e1; e += 32) {
            int32_t c = (e + lane < e1) ? szcol[e + lane] : 0;
            bool keep = (e + lane < e1) && hz[c] < 0;
            unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) slcol[base + __popc(m & ((1u << lane) - 1u))] = c;
            base += __popc(m);
        }
    }
}

__global__ void to_i32_kernel(const uint32_t* in, int64_t n, int32_t* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)in[i];
}

}  // namespace

int64_t heavy_ids(const int32_t* deg_a, const int32_t* deg_b, int64_t n, int64_t thr,
                  int32_t* h, int32_t* h_inv, Arena& ws, cudaStream_t st) {
    if (n <= 0) return 0;
    uint32_t* flag = ws.get<uint32_t>(n);
    uint32_t* idx = ws.get<uint32_t>(n);
    uint32_t* d_cnt = ws.get<uint32_t>(1);
    heavy_flag_kernel<<<G(n), 256, 0, st>>>(deg_a, deg_b, n, thr, flag);
    JP_CHECK_LAUNCH();
    scan_u32(flag, idx, n, d_cnt, ws, st);
    heavy_assign_kernel<<<G(n), 256, 0, st>>>(flag, idx, n, h, h_inv);
    JP_CHECK_LAUNCH();
    uint32_t c = 0;
    JP_CUDA_TRY(cudaMemcpyAsync(&c, d_cnt, sizeof(c), cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaStreamSynchronize(st));
    return c;
}

void build_partition(const Graph& g, Partition& p, Arena& ws, cudaStream_t st,
                     int64_t* host_scalars) {
    (void)host_scalars;
    p.hx = ws.get<int32_t>(g.nx + 1);
    p.hx_inv = ws.get<int32_t>(g.nx + 1);
    p.u = heavy_ids(g.deg_rx, nullptr, g.nx, p.d2, p.hx, p.hx_inv, ws, st);
    p.hy = ws.get<int32_t>(g.ny + 1);
    p.hy_inv = ws.get<int32_t>(g.ny + 1);
    p.v = heavy_ids(g.deg_ry, g.self ? nullptr : g.deg_sy, g.ny, p.d1, p.hy, p.hy_inv, ws, st);
    if (g.self) {
        p.hz = p.hx;
        p.hz_inv = p.hx_inv;
        p.w = p.u;
    } else {
        p.hz = ws.get<int32_t>(g.nz + 1);
        p.hz_inv = ws.get<int32_t>(g.nz + 1);
        p.w = heavy_ids(g.deg_sz, nullptr, g.nz, p.d2, p.hz, p.hz_inv, ws, st);
    }
    build_light_z_lists(g.syoff, g.szcol, p, ws, st);
}

void build_light_z_lists(const int32_t* syoff, const int32_t* szcol, Partition& p, Arena& ws,
                         cudaStream_t st) {
    p.sloff = ws.get<int32_t>(p.v + 2);
    uint32_t* cnt = ws.get<uint32_t>(p.v + 1);
    uint32_t* off = ws.get<uint32_t>(p.v + 1);
    uint32_t* d_tot = ws.get<uint32_t>(1);
    if (p.v > 0) {
        light_z_count_kernel<<<grid_for(p.v * 32, 256, 152 * 16), 256, 0, st>>>(
            p.hy_inv, p.v, syoff, szcol, p.hz, cnt);
        JP_CHECK_LAUNCH();
    }
    scan_u32(cnt, off, p.v, d_tot, ws, st);
    uint32_t tot = 0;
    JP_CUDA_TRY(cudaMemcpyAsync(&tot, d_tot, sizeof(tot), cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaStreamSynchronize(st));
    p.slcol = ws.get<int32_t>((int64_t)tot + 1);
    if (p.v > 0) {
        light_z_fill_kernel<<<grid_for(p.v * 32, 256, 152 * 16), 256, 0, st>>>(
            p.hy_inv, p.v, syoff, szcol, p.hz, off, p.slcol);
        JP_CHECK_LAUNCH();
        to_i32_kernel<<<G(p.v), 256, 0, st>>>(off, p.v, p.sloff);
        JP_CHECK_LAUNCH();
    }
    JP_CUDA_TRY(cudaMemcpyAsync(p.sloff + p.v, d_tot, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
}

}  // namespace jp
