// Normalisation and index building (Section 5, "Indexing relations").
//
// Relations are sets: duplicate tuples are removed.  Values are dictionary
// encoded to dense ids in sorted value order, so sorting by id equals sorting
// by signed value.  R is indexed by x (CSR: x -> sorted y ids) and S by y
// (CSR: y -> sorted z ids); the degree arrays and the full join size
// |OUT_join| = sum_y deg_R(y) deg_S(y) follow in one linear pass.  Tuples of R
// whose y does not occur in S cannot contribute and are dropped (the
// dangling-tuple removal of Section 3.1).
#include "jp_internal.cuh"

namespace jp {
namespace {

constexpr uint32_t BIAS = 0x80000000u;

__device__ __forceinline__ int32_t unbias(uint32_t v) { return (int32_t)(v ^ BIAS); }

__global__ void pack_keys_kernel(const int32_t* a, const int32_t* b, int64_t n, uint64_t* keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t hi = (uint32_t)a[i] ^ BIAS;
        uint32_t lo = (uint32_t)b[i] ^ BIAS;
        keys[i] = ((uint64_t)hi << 32) | lo;
    }
}

// keys from a single column (upper half zero)
__global__ void pack_lo_kernel(const int32_t* a, int64_t n, uint64_t* keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = (uint64_t)((uint32_t)a[i] ^ BIAS);
}

__global__ void swap_halves_kernel(const uint64_t* in, int64_t n, uint64_t* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = in[i];
        out[i] = (k << 32) | (k >> 32);
    }
}

__global__ void run_flag_kernel(const uint64_t* k, int64_t n, uint32_t* flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || (k[i] >> 32) != (k[i - 1] >> 32)) ? 1u : 0u;
}

__global__ void run_emit_kernel(const uint64_t* k, int64_t n, const uint32_t* gid, int32_t* gval,
                                int32_t* goff, int32_t* lo) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t key = k[i];
        if (i == 0 || (key >> 32) != (k[i - 1] >> 32)) {
            gval[gid[i]] = unbias((uint32_t)(key >> 32));
            goff[gid[i]] = (int32_t)i;
        }
        if (lo) lo[i] = unbias((uint32_t)key);
    }
}

__global__ void set_tail_kernel(int32_t* goff, const uint32_t* d_g, int32_t n) {
    goff[*d_g] = n;
}

__global__ void unbias_lo_kernel(const uint64_t* k, int64_t n, int32_t* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = unbias((uint32_t)k[i]);
}

// id[i] = position of q[i] in the sorted dictionary, or -1 if absent
__global__ void lookup_kernel(const int32_t* dict, int64_t nd, const int32_t* q, int64_t n,
                              int32_t* id) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = q[i];
        int64_t lo = 0, hi = nd;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (dict[mid] < v) lo = mid + 1; else hi = mid;
        }
        id[i] = (lo < nd && dict[lo] == v) ? (int32_t)lo : -1;
    }
}

__global__ void keep_flag_kernel(const int32_t* id, int64_t n, uint32_t* flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = id[i] >= 0 ? 1u : 0u;
}

__global__ void keep_scatter_kernel(const uint64_t* k, const int32_t* id, int64_t n,
                                    const uint32_t* pos, uint64_t* k_out, int32_t* id_out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (id[i] >= 0) {
            k_out[pos[i]] = k[i];
            id_out[pos[i]] = id[i];
        }
}

__global__ void deg_from_off_kernel(const int32_t* off, int64_t n, int32_t* deg) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        deg[i] = off[i + 1] - off[i];
}

__global__ void deg_hist_kernel(const int32_t* col, int64_t n, int32_t* deg) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&deg[col[i]], 1);
}

__global__ void out_join_kernel(const int32_t* a, const int32_t* b, int64_t n,
                                unsigned long long* acc) {
    unsigned long long s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        s += (unsigned long long)a[i] * (unsigned long long)b[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(acc, s);
}

// xsum[a] = sum over the y of R[a] of deg_S(y): lane per x; the x of a warp
// with more than 32 neighbours are summed by the whole warp, one after another
__global__ void xsum_kernel(int64_t nx, const int32_t* __restrict__ rxoff,
                            const int32_t* __restrict__ rycol, const int32_t* __restrict__ deg_sy,
                            int64_t* __restrict__ xsum) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; base < nx;
         base += stride) {
        const int64_t a = base + lane;
        const bool valid = a < nx;
        int32_t e0 = 0, e1 = 0;
        if (valid) {
            e0 = rxoff[a];
            e1 = rxoff[a + 1];
        }
        const bool small = valid && e1 - e0 <= 32;
        long long c = 0;
        if (small) {
            int32_t e = e0;
            for (; e + 4 <= e1; e += 4) {
                const int32_t b0 = rycol[e], b1 = rycol[e + 1], b2 = rycol[e + 2], b3 = rycol[e + 3];
                c += (long long)deg_sy[b0] + deg_sy[b1] + deg_sy[b2] + deg_sy[b3];
            }
            for (; e < e1; ++e) c += deg_sy[rycol[e]];
        }
        unsigned big = __ballot_sync(0xffffffffu, valid && !small);
        while (big) {
            const int j = __ffs(big) - 1;
            big &= big - 1;
            const int32_t f0 = __shfl_sync(0xffffffffu, e0, j), f1 = __shfl_sync(0xffffffffu, e1, j);
            long long sj = 0;
            int32_t e = f0 + lane;
            for (; e + 7 * 32 < f1; e += 8 * 32) {
                int32_t b[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) b[u] = rycol[e + 32 * u];
#pragma unroll
                for (int u = 0; u < 8; ++u) sj += deg_sy[b[u]];
            }
            for (; e < f1; e += 32) sj += deg_sy[rycol[e]];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sj += __shfl_xor_sync(0xffffffffu, sj, o);
            if (lane == j) c = sj;
        }
        if (valid) xsum[a] = (int64_t)c;
    }
}

inline int G(int64_t n) { return grid_for(n, 256, 152 * 16); }

// Sort + unique 64-bit keys; returns the unique keys buffer and count.
uint64_t* sort_unique(uint64_t* keys, uint64_t* tmp, int64_t n, int64_t* count, Arena& ws,
                      cudaStream_t st, uint32_t* hist_host, int64_t* host_scalars) {
    uint64_t* sorted = radix_sort_u64(keys, tmp, n, ws, st, hist_host);
    uint64_t* out = (sorted == keys) ? tmp : keys;
    uint32_t* d_cnt = ws.get<uint32_t>(1);
    unique_u64(sorted, n, out, d_cnt, ws, st);
    uint32_t c = 0;
    JP_CUDA_TRY(cudaMemcpyAsync(&c, d_cnt, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaStreamSynchronize(st));
    *count = c;
    (void)host_scalars;
    return out;
}

// Group sorted keys by their upper half.
void runs_hi(const uint64_t* keys, int64_t n, int32_t* gval, int32_t* goff, int32_t* lo,
             uint32_t* d_g, Arena& ws, cudaStream_t st) {
    uint32_t* flag = ws.get<uint32_t>(n > 0 ? n : 1);
    uint32_t* gid = ws.get<uint32_t>(n > 0 ? n : 1);
    if (n > 0) {
        run_flag_kernel<<<G(n), 256, 0, st>>>(keys, n, flag);
        JP_CHECK_LAUNCH();
    }
    scan_u32(flag, gid, n, d_g, ws, st);
    if (n > 0) {
        run_emit_kernel<<<G(n), 256, 0, st>>>(keys, n, gid, gval, goff, lo);
        JP_CHECK_LAUNCH();
    }
    set_tail_kernel<<<1, 1, 0, st>>>(goff, d_g, (int32_t)n);
    JP_CHECK_LAUNCH();
}

uint32_t read_u32(const uint32_t* d, cudaStream_t st) {
    uint32_t v = 0;
    JP_CUDA_TRY(cudaMemcpyAsync(&v, d, sizeof(v), cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaStreamSynchronize(st));
    return v;
}

}  // namespace

void build_graph(const jp_rel* R, const jp_rel* S, Graph& g, Arena& ws, cudaStream_t st,
                 uint32_t* d_status, uint32_t* hist_host, int64_t* host_scalars) {
    (void)d_status;
    const int64_t n = R->n;
    g.self = (S == nullptr);
    // ---- R: distinct (x, y), sorted by (x, y)
    uint64_t* k0 = ws.get<uint64_t>(n > 0 ? n : 1);
    uint64_t* k1 = ws.get<uint64_t>(n > 0 ? n : 1);
    if (n > 0) {
        pack_keys_kernel<<<G(n), 256, 0, st>>>(R->x, R->y, n, k0);
        JP_CHECK_LAUNCH();
    }
    int64_t nr0 = 0;
    uint64_t* ur = sort_unique(k0, k1, n, &nr0, ws, st, hist_host, host_scalars);
    uint64_t* spare = (ur == k0) ? k1 : k0;

    if (g.self) {
        g.nr = g.ns = nr0;
        // x runs of R
        g.xval = ws.get<int32_t>(nr0 + 1);
        g.rxoff = ws.get<int32_t>(nr0 + 2);
        int32_t* ry_val = ws.get<int32_t>(nr0 + 1);
        uint32_t* d_nx = ws.get<uint32_t>(1);
        runs_hi(ur, nr0, g.xval, g.rxoff, ry_val, d_nx, ws, st);
        // S = R indexed by y: keys (y, x)
        if (nr0 > 0) {
            swap_halves_kernel<<<G(nr0), 256, 0, st>>>(ur, nr0, spare);
            JP_CHECK_LAUNCH();
        }
        uint64_t* spare2 = ws.get<uint64_t>(nr0 > 0 ? nr0 : 1);
        uint64_t* ys = radix_sort_u64(spare, spare2, nr0, ws, st, hist_host);
        g.yval = ws.get<int32_t>(nr0 + 1);
        g.syoff = ws.get<int32_t>(nr0 + 2);
        int32_t* sx_val = ws.get<int32_t>(nr0 + 1);
        uint32_t* d_ny = ws.get<uint32_t>(1);
        runs_hi(ys, nr0, g.yval, g.syoff, sx_val, d_ny, ws, st);
        g.nx = read_u32(d_nx, st);
        g.ny = read_u32(d_ny, st);
        g.nz = g.nx;
        g.zval = g.xval;
        g.rycol = ws.get<int32_t>(nr0 + 1);
        g.szcol = ws.get<int32_t>(nr0 + 1);
        if (nr0 > 0) {
            lookup_kernel<<<G(nr0), 256, 0, st>>>(g.yval, g.ny, ry_val, nr0, g.rycol);
            JP_CHECK_LAUNCH();
            lookup_kernel<<<G(nr0), 256, 0, st>>>(g.xval, g.nx, sx_val, nr0, g.szcol);
            JP_CHECK_LAUNCH();
        }
        g.deg_rx = ws.get<int32_t>(g.nx + 1);
        g.deg_sy = ws.get<int32_t>(g.ny + 1);
        if (g.nx > 0) { deg_from_off_kernel<<<G(g.nx), 256, 0, st>>>(g.rxoff, g.nx, g.deg_rx); JP_CHECK_LAUNCH(); }
        if (g.ny > 0) { deg_from_off_kernel<<<G(g.ny), 256, 0, st>>>(g.syoff, g.ny, g.deg_sy); JP_CHECK_LAUNCH(); }
        g.deg_ry = g.deg_sy;
        g.deg_sz = g.deg_rx;
    } else {
        const int64_t m = S->n;
        // ---- S: distinct (z, y), sorted by (y, z)
        uint64_t* s0 = ws.get<uint64_t>(m > 0 ? m : 1);
        uint64_t* s1 = ws.get<uint64_t>(m > 0 ? m : 1);
        if (m > 0) {
            pack_keys_kernel<<<G(m), 256, 0, st>>>(S->y, S->x, m, s0);
            JP_CHECK_LAUNCH();
        }
        int64_t ns = 0;
        uint64_t* us = sort_unique(s0, s1, m, &ns, ws, st, hist_host, host_scalars);
        uint64_t* sspare = (us == s0) ? s1 : s0;
        g.ns = ns;
        g.yval = ws.get<int32_t>(ns + 1);
        g.syoff = ws.get<int32_t>(ns + 2);
        int32_t* sz_val = ws.get<int32_t>(ns + 1);
        uint32_t* d_ny = ws.get<uint32_t>(1);
        runs_hi(us, ns, g.yval, g.syoff, sz_val, d_ny, ws, st);
        // z dictionary: distinct z values of S
        if (ns > 0) {
            pack_lo_kernel<<<G(ns), 256, 0, st>>>(sz_val, ns, sspare);
            JP_CHECK_LAUNCH();
        }
        uint64_t* zt = ws.get<uint64_t>(ns > 0 ? ns : 1);
        int64_t nz = 0;
        uint64_t* uz = sort_unique(sspare, zt, ns, &nz, ws, st, hist_host, host_scalars);
        g.nz = nz;
        g.zval = ws.get<int32_t>(nz + 1);
        if (nz > 0) {
            unbias_lo_kernel<<<G(nz), 256, 0, st>>>(uz, nz, g.zval);
            JP_CHECK_LAUNCH();
        }
        g.ny = read_u32(d_ny, st);
        g.szcol = ws.get<int32_t>(ns + 1);
        if (ns > 0) {
            lookup_kernel<<<G(ns), 256, 0, st>>>(g.zval, g.nz, sz_val, ns, g.szcol);
            JP_CHECK_LAUNCH();
        }
        // ---- R: drop tuples whose y has no S tuple, then index by x
        int32_t* ry_val = ws.get<int32_t>(nr0 + 1);
        int32_t* ry_id = ws.get<int32_t>(nr0 + 1);
        if (nr0 > 0) {
            unbias_lo_kernel<<<G(nr0), 256, 0, st>>>(ur, nr0, ry_val);
            JP_CHECK_LAUNCH();
            lookup_kernel<<<G(nr0), 256, 0, st>>>(g.yval, g.ny, ry_val, nr0, ry_id);
            JP_CHECK_LAUNCH();
        }
        uint32_t* flag = ws.get<uint32_t>(nr0 + 1);
        uint32_t* pos = ws.get<uint32_t>(nr0 + 1);
        uint32_t* d_nr = ws.get<uint32_t>(1);
        if (nr0 > 0) {
            keep_flag_kernel<<<G(nr0), 256, 0, st>>>(ry_id, nr0, flag);
            JP_CHECK_LAUNCH();
        }
        scan_u32(flag, pos, nr0, d_nr, ws, st);
        g.rycol = ws.get<int32_t>(nr0 + 1);
        if (nr0 > 0) {
            keep_scatter_kernel<<<G(nr0), 256, 0, st>>>(ur, ry_id, nr0, pos, spare, g.rycol);
            JP_CHECK_LAUNCH();
        }
        g.nr = read_u32(d_nr, st);
        g.xval = ws.get<int32_t>(g.nr + 1);
        g.rxoff = ws.get<int32_t>(g.nr + 2);
        uint32_t* d_nx = ws.get<uint32_t>(1);
        runs_hi(spare, g.nr, g.xval, g.rxoff, nullptr, d_nx, ws, st);
        g.nx = read_u32(d_nx, st);
        g.deg_rx = ws.get<int32_t>(g.nx + 1);
        g.deg_sy = ws.get<int32_t>(g.ny + 1);
        g.deg_ry = ws.get<int32_t>(g.ny + 1);
        g.deg_sz = ws.get<int32_t>(g.nz + 1);
        JP_CUDA_TRY(cudaMemsetAsync(g.deg_ry, 0, (g.ny + 1) * sizeof(int32_t), st));
        JP_CUDA_TRY(cudaMemsetAsync(g.deg_sz, 0, (g.nz + 1) * sizeof(int32_t), st));
        if (g.nx > 0) { deg_from_off_kernel<<<G(g.nx), 256, 0, st>>>(g.rxoff, g.nx, g.deg_rx); JP_CHECK_LAUNCH(); }
        if (g.ny > 0) { deg_from_off_kernel<<<G(g.ny), 256, 0, st>>>(g.syoff, g.ny, g.deg_sy); JP_CHECK_LAUNCH(); }
        if (g.nr > 0) { deg_hist_kernel<<<G(g.nr), 256, 0, st>>>(g.rycol, g.nr, g.deg_ry); JP_CHECK_LAUNCH(); }
        if (g.ns > 0) { deg_hist_kernel<<<G(g.ns), 256, 0, st>>>(g.szcol, g.ns, g.deg_sz); JP_CHECK_LAUNCH(); }
    }
    // every x's join candidates, read by threshold selection and by the light
    // part's classification
    g.xsum = ws.get<int64_t>(g.nx + 1);
    if (g.nx > 0) {
        xsum_kernel<<<grid_for(g.nx, 256, 152 * 16), 256, 0, st>>>(g.nx, g.rxoff, g.rycol, g.deg_sy,
                                                                  g.xsum);
        JP_CHECK_LAUNCH();
    }
    // |OUT_join| = sum_y deg_R(y) deg_S(y)
    unsigned long long* acc = ws.get<unsigned long long>(1);
    JP_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(unsigned long long), st));
    if (g.ny > 0) {
        out_join_kernel<<<G(g.ny), 256, 0, st>>>(g.deg_ry, g.deg_sy, g.ny, acc);
        JP_CHECK_LAUNCH();
    }
    unsigned long long oj = 0;
    JP_CUDA_TRY(cudaMemcpyAsync(&oj, acc, sizeof(oj), cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaStreamSynchronize(st));
    g.out_join = (double)oj;
}

}  // namespace jp
