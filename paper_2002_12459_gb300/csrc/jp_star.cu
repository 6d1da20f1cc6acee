// Star query Q*_3(x1,x2,x3) = R1(x1,y), R2(x2,y), R3(x3,y) (Section 2.1,
// Section 3.2).
//
// The witnesses are factorised on (x1, x2): for every pair (a1, a2) the set
// B(a1,a2) = {b : (a1,b) in R1, (a2,b) in R2} is formed (the triples
// (a1, a2, b) are enumerated from R1 by x and R2 by y, then sorted), and the
// output of the pair is the union of R3[b] over b in B(a1,a2).  Each pair is
// one "row" of a virtual two-path instance whose neighbour lists are the b's
// of B and whose S is R3 indexed by y, so the light expansion, the
// deduplication, the heavy product and the output placement of the two-path
// pipeline apply unchanged:
//   - light/heavy split of Section 3.2: x_i is heavy when deg_Ri(x_i) >
//     Delta2; y is heavy when at least two relations give it degree > Delta1
//     (a tuple (a_i, b) is in R_i^diamond iff every other relation gives b
//     degree <= Delta1, so a witness is left to the product iff all a_i are
//     heavy and no (a_i, b) is in R_i^diamond);
//   - the heavy pairs (a1, a2) (both heavy) are the rows of V, the heavy x3
//     the rows of W, the heavy y the shared columns (ceil(3/2) = 2 variables
//     on the V side, floor(3/2) = 1 on the W side); V x W^T runs on the
//     tensor cores and its bitmap is united with the light lists of the
//     heavy pairs;
//   - the light lists of a heavy pair take, from a heavy b, only the light
//     x3 of R3[b].
// Relations with a single y value list per pair need no deduplication at all
// (the copy fast path of the light pass).
#include <algorithm>
#include <cmath>

#include "jp_internal.cuh"

namespace jp {
namespace {

constexpr uint32_t BIAS = 0x80000000u;
inline int G(int64_t n) { return grid_for(n, 256, 152 * 16); }

__global__ void pack_kernel(const int32_t* hi, const int32_t* lo, int64_t n, uint64_t* keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = ((uint64_t)((uint32_t)hi[i] ^ BIAS) << 32) | (uint32_t)((uint32_t)lo[i] ^ BIAS);
}

__global__ void split_kernel(const uint64_t* keys, int64_t n, int32_t* hi, int32_t* lo) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        if (hi) hi[i] = (int32_t)((uint32_t)(k >> 32) ^ BIAS);
        if (lo) lo[i] = (int32_t)((uint32_t)k ^ BIAS);
    }
}

// keys holding one biased value in the low half
__global__ void pack_one_kernel(const int32_t* v, int64_t n, uint64_t* keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = (uint64_t)((uint32_t)v[i] ^ BIAS);
}

__global__ void lookup_kernel(const int32_t* dict, int64_t nd, const int32_t* q, int64_t n,
                              int32_t* id) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = q[i];
        int64_t lo = 0, hi = nd;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (dict[mid] < v) lo = mid + 1; else hi = mid;
        }
        id[i] = (lo < nd && dict[lo] == v) ? (int32_t)lo : -1;
    }
}

__global__ void hist_kernel(const int32_t* col, int64_t n, int32_t* cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (col[i] >= 0) atomicAdd(&cnt[col[i]], 1);
}

__global__ void keep_kernel(const int32_t* yid, const int32_t* xv, int64_t n, const uint32_t* pos,
                            int32_t* yid_out, int32_t* xv_out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (yid[i] >= 0) {
            yid_out[pos[i]] = yid[i];
            xv_out[pos[i]] = xv[i];
        }
}

__global__ void flag_nonneg_kernel(const int32_t* v, int64_t n, uint32_t* flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = v[i] >= 0 ? 1u : 0u;
}

__global__ void run_start_kernel(const uint64_t* k, int64_t n, int shift, uint32_t* flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || (k[i] >> shift) != (k[i - 1] >> shift)) ? 1u : 0u;
}

// value dictionary from sorted unique keys (low half) and row offsets
__global__ void unbias_lo_kernel(const uint64_t* k, int64_t n, int32_t* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)((uint32_t)k[i] ^ BIAS);
}

__global__ void x_runs_kernel(const uint64_t* k, int64_t n, const uint32_t* gid, int32_t* xval,
                              int32_t* xoff) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (i == 0 || (k[i] >> 32) != (k[i - 1] >> 32)) {
            xval[gid[i]] = (int32_t)((uint32_t)(k[i] >> 32) ^ BIAS);
            xoff[gid[i]] = (int32_t)i;
        }
}

__global__ void set_last_kernel(int32_t* arr, const uint32_t* d_idx, int32_t v) {
    arr[*d_idx] = v;
}

__global__ void deg_off_kernel(const int32_t* off, int64_t n, int32_t* deg) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        deg[i] = off[i + 1] - off[i];
}

// number of (a1, a2, b) triples each R1 tuple produces
__global__ void triple_count_kernel(const int32_t* r1ycol, int64_t n1, const int32_t* deg2y,
                                    const int32_t* deg3y, int64_t* cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n1;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = r1ycol[i];
        cnt[i] = deg3y[b] > 0 ? deg2y[b] : 0;
    }
}

// warp per a1 row of R1: key (a1 | a2 | b) for every a2 in R2[b]
__global__ void triple_fill_kernel(int64_t nx1, const int32_t* r1off, const int32_t* r1ycol,
                                   const int64_t* toff, const int32_t* r2off,
                                   const int32_t* r2col, const int32_t* deg3y, int sh1, int sh2,
                                   uint64_t* keys) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a1 = warp; a1 < nx1; a1 += nwarps) {
        for (int32_t e = r1off[a1]; e < r1off[a1 + 1]; ++e) {
            const int32_t b = r1ycol[e];
            if (deg3y[b] == 0) continue;
            const int64_t o = toff[e];
            const int32_t s0 = r2off[b], L = r2off[b + 1] - s0;
            for (int32_t t = lane; t < L; t += 32)
                keys[o + t] = ((uint64_t)a1 << sh1) | ((uint64_t)r2col[s0 + t] << sh2) | (uint64_t)b;
        }
    }
}

__global__ void group_emit_kernel(const uint64_t* keys, int64_t n, const uint32_t* gid, int sh1,
                                  int sh2, uint64_t m2, uint64_t my, int32_t* ga1, int32_t* ga2,
                                  int32_t* goff, int32_t* bcol) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        if (i == 0 || (k >> sh2) != (keys[i - 1] >> sh2)) {
            const uint32_t g = gid[i];
            ga1[g] = (int32_t)(k >> sh1);
            ga2[g] = (int32_t)((k >> sh2) & m2);
            goff[g] = (int32_t)i;
        }
        bcol[i] = (int32_t)(k & my);
    }
}

// pd[g] = 1 iff both a1 and a2 of the pair are heavy
__global__ void pair_heavy_kernel(const int32_t* ga1, const int32_t* ga2, int64_t ng,
                                  const int32_t* deg1x, const int32_t* deg2x, int64_t d2,
                                  int32_t* pd) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng;
         g += (int64_t)gridDim.x * blockDim.x)
        pd[g] = (deg1x[ga1[g]] > d2 && deg2x[ga2[g]] > d2) ? 1 : 0;
}

// number of relations giving y degree > d1
__global__ void y_heavy_count_kernel(const int32_t* d1y, const int32_t* d2y, const int32_t* d3y,
                                     int64_t ny, int64_t d1, int32_t* cnt) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < ny;
         b += (int64_t)gridDim.x * blockDim.x)
        cnt[b] = (d1y[b] > d1) + (d2y[b] > d1) + (d3y[b] > d1);
}

__global__ void gather_vals_kernel(const int32_t* ids, int64_t n, const int32_t* val, int32_t* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = val[ids[i]];
}

__global__ void star_join_kernel(const int32_t* d1y, const int32_t* d2y, const int32_t* d3y,
                                 int64_t ny, unsigned long long* acc) {
    unsigned long long s = 0;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < ny;
         b += (int64_t)gridDim.x * blockDim.x)
        s += (unsigned long long)d1y[b] * (unsigned long long)d2y[b] * (unsigned long long)d3y[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(acc, s);
}

template <typename T>
T read1(const T* d, cudaStream_t st) {
    T v;
    JP_CUDA_TRY(cudaMemcpyAsync(&v, d, sizeof(T), cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaStreamSynchronize(st));
    return v;
}

int bits_for(int64_t n) {
    int b = 1;
    while (b < 62 && ((int64_t)1 << b) < n) ++b;
    return b;
}

// Sorted distinct values of v[0..n) -> dict (returns its size).
int64_t make_dict(const int32_t* v, int64_t n, int32_t** dict, Arena& ws, cudaStream_t st,
                  uint32_t* hist_host) {
    uint64_t* k0 = ws.get<uint64_t>(n > 0 ? n : 1);
    uint64_t* k1 = ws.get<uint64_t>(n > 0 ? n : 1);
    if (n > 0) {
        pack_one_kernel<<<G(n), 256, 0, st>>>(v, n, k0);
        JP_CHECK_LAUNCH();
    }
    uint64_t* s = radix_sort_u64(k0, k1, n, ws, st, hist_host);
    uint64_t* u = (s == k0) ? k1 : k0;
    uint32_t* d_cnt = ws.get<uint32_t>(1);
    unique_u64(s, n, u, d_cnt, ws, st);
    const int64_t nd = read1(d_cnt, st);
    *dict = ws.get<int32_t>(nd + 1);
    if (nd > 0) {
        unbias_lo_kernel<<<G(nd), 256, 0, st>>>(u, nd, *dict);
        JP_CHECK_LAUNCH();
    }
    return nd;
}

// One relation indexed by y over the shared y dictionary: CSR off[ny+1] of
// x ids (sorted within a y), x dictionary, degrees.  Tuples whose y is not in
// the dictionary cannot join and are dropped.
struct ByY {
    int64_t n = 0, nx = 0;
    int32_t* xval = nullptr;
    int32_t* off = nullptr;
    int32_t* col = nullptr;
    int32_t* degx = nullptr;
    int32_t* degy = nullptr;
};

void index_by_y(const jp_rel* R, const int32_t* yval, int64_t ny, ByY& out, Arena& ws,
                cudaStream_t st, uint32_t* hist_host) {
    const int64_t n = R->n;
    uint64_t* k0 = ws.get<uint64_t>(n > 0 ? n : 1);
    uint64_t* k1 = ws.get<uint64_t>(n > 0 ? n : 1);
    if (n > 0) {
        pack_kernel<<<G(n), 256, 0, st>>>(R->y, R->x, n, k0);
        JP_CHECK_LAUNCH();
    }
    uint64_t* s = radix_sort_u64(k0, k1, n, ws, st, hist_host);
    uint64_t* u = (s == k0) ? k1 : k0;
    uint32_t* d_cnt = ws.get<uint32_t>(1);
    unique_u64(s, n, u, d_cnt, ws, st);
    const int64_t m = read1(d_cnt, st);
    int32_t* yv = ws.get<int32_t>(m + 1);
    int32_t* xv = ws.get<int32_t>(m + 1);
    int32_t* yid = ws.get<int32_t>(m + 1);
    if (m > 0) {
        split_kernel<<<G(m), 256, 0, st>>>(u, m, yv, xv);
        JP_CHECK_LAUNCH();
        lookup_kernel<<<G(m), 256, 0, st>>>(yval, ny, yv, m, yid);
        JP_CHECK_LAUNCH();
    }
    uint32_t* flag = ws.get<uint32_t>(m + 1);
    uint32_t* pos = ws.get<uint32_t>(m + 1);
    uint32_t* d_kept = ws.get<uint32_t>(1);
    if (m > 0) {
        flag_nonneg_kernel<<<G(m), 256, 0, st>>>(yid, m, flag);
        JP_CHECK_LAUNCH();
    }
    scan_u32(flag, pos, m, d_kept, ws, st);
    const int64_t kept = read1(d_kept, st);
    int32_t* kyid = ws.get<int32_t>(kept + 1);
    int32_t* kxv = ws.get<int32_t>(kept + 1);
    if (m > 0) {
        keep_kernel<<<G(m), 256, 0, st>>>(yid, xv, m, pos, kyid, kxv);
        JP_CHECK_LAUNCH();
    }
    out.n = kept;
    out.nx = make_dict(kxv, kept, &out.xval, ws, st, hist_host);
    out.col = ws.get<int32_t>(kept + 1);
    if (kept > 0) {
        lookup_kernel<<<G(kept), 256, 0, st>>>(out.xval, out.nx, kxv, kept, out.col);
        JP_CHECK_LAUNCH();
    }
    out.degy = ws.get<int32_t>(ny + 1);
    out.degx = ws.get<int32_t>(out.nx + 1);
    JP_CUDA_TRY(cudaMemsetAsync(out.degy, 0, (ny + 1) * sizeof(int32_t), st));
    JP_CUDA_TRY(cudaMemsetAsync(out.degx, 0, (out.nx + 1) * sizeof(int32_t), st));
    if (kept > 0) {
        hist_kernel<<<G(kept), 256, 0, st>>>(kyid, kept, out.degy);
        JP_CHECK_LAUNCH();
        hist_kernel<<<G(kept), 256, 0, st>>>(out.col, kept, out.degx);
        JP_CHECK_LAUNCH();
    }
    // offsets: exclusive scan of the y degrees (tuples are sorted by y id)
    out.off = ws.get<int32_t>(ny + 2);
    uint32_t* d_tot = ws.get<uint32_t>(1);
    scan_u32(reinterpret_cast<const uint32_t*>(out.degy), reinterpret_cast<uint32_t*>(out.off), ny,
             d_tot, ws, st);
    JP_CUDA_TRY(cudaMemcpyAsync(out.off + ny, d_tot, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
}

// Section 3.2 cost with omega = 2 and the Lemma 1 rectangular product:
// N D1^(k-1) + OUT D2 + M((N/D2)^ceil(k/2), N/D1, (N/D2)^floor(k/2)).
double star_cost(double N, double OUT, double d1, double d2, int k) {
    const int kv = (k + 1) / 2, kw = k / 2;
    const double U = std::pow(N / d2, kv), V = N / d1, W = std::pow(N / d2, kw);
    const double beta = std::min(U, std::min(V, W));
    return N * std::pow(d1, k - 1) + OUT * d2 + U * V * W / beta;
}

// ---- star queries with k > 3: the tail relations grouped on y
// triples per y of two relations P, Q: degP(b) * degQ(b)
__global__ void pair_count_kernel(const int32_t* dp, const int32_t* dq, int64_t ny, int64_t* cnt) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < ny;
         b += (int64_t)gridDim.x * blockDim.x)
        cnt[b] = (int64_t)dp[b] * dq[b];
}

// warp per y: key (p | q | b) for every p in P[b] and q in Q[b]
__global__ void pair_fill_kernel(int64_t ny, const int32_t* poff, const int32_t* pcol,
                                 const int32_t* qoff, const int32_t* qcol, const int64_t* toff,
                                 int shp, int shq, uint64_t* keys) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = warp; b < ny; b += nwarps) {
        const int32_t p0 = poff[b], dp = poff[b + 1] - p0;
        const int32_t q0 = qoff[b], dq = qoff[b + 1] - q0;
        const int64_t n = (int64_t)dp * dq, o = toff[b];
        for (int64_t t = lane; t < n; t += 32) {
            const int64_t i = t / dq, j = t - i * dq;
            keys[o + t] = ((uint64_t)pcol[p0 + i] << shp) | ((uint64_t)qcol[q0 + j] << shq) |
                          (uint64_t)b;
        }
    }
}

// one tuple (g, y value) per sorted triple; the pair's values at its first
// triple.  gid is the exclusive scan of the group-start flags, so a triple
// after its group's first one has gid = g + 1.
__global__ void pair_emit_kernel(const uint64_t* keys, int64_t n, const uint32_t* gid, int shp,
                                 int shq, uint64_t mq, uint64_t my, const int32_t* pval,
                                 const int32_t* qval, const int32_t* yval, int32_t* gx,
                                 int32_t* gy, int32_t* gp, int32_t* gq) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        const bool start = i == 0 || (k >> shq) != (keys[i - 1] >> shq);
        const uint32_t g = start ? gid[i] : gid[i] - 1u;
        if (start) {
            gp[g] = pval[k >> shp];
            gq[g] = qval[(k >> shq) & mq];
        }
        gx[i] = (int32_t)g;
        gy[i] = yval[k & my];
    }
}

}  // namespace

// Minimiser of the star cost over a log-spaced grid of integer thresholds.
void star_thresholds(int64_t N, double out_est, int k, int64_t* d1, int64_t* d2) {
    const int steps = 96;
    double best = INFINITY;
    int64_t b1 = 1, b2 = 1;
    const double lnN = std::log((double)std::max<int64_t>(N, 1));
    for (int i = 0; i <= steps; ++i) {
        const int64_t t1 = std::max<int64_t>(1, (int64_t)std::floor(std::exp(lnN * i / steps)));
        for (int j = 0; j <= steps; ++j) {
            const int64_t t2 = std::max<int64_t>(1, (int64_t)std::floor(std::exp(lnN * j / steps)));
            const double c = star_cost((double)N, out_est, (double)t1, (double)t2, k);
            if (c < best) {
                best = c;
                b1 = t1;
                b2 = t2;
            }
        }
    }
    *d1 = b1;
    *d2 = b2;
}

void run_star3(const jp_rel* rels, int mode, int64_t fd1, int64_t fd2, StarOut& so, Arena& ws,
               cudaStream_t st, uint32_t* d_status, uint32_t* hist_host) {
    // ---- R1 indexed by x, shared y dictionary from R1
    const jp_rel* R1 = &rels[0];
    const int64_t n = R1->n;
    uint64_t* k0 = ws.get<uint64_t>(n > 0 ? n : 1);
    uint64_t* k1 = ws.get<uint64_t>(n > 0 ? n : 1);
    if (n > 0) {
        pack_kernel<<<G(n), 256, 0, st>>>(R1->x, R1->y, n, k0);
        JP_CHECK_LAUNCH();
    }
    uint64_t* s = radix_sort_u64(k0, k1, n, ws, st, hist_host);
    uint64_t* u1 = (s == k0) ? k1 : k0;
    uint32_t* d_cnt = ws.get<uint32_t>(1);
    unique_u64(s, n, u1, d_cnt, ws, st);
    const int64_t n1 = read1(d_cnt, st);
    int32_t* r1y = ws.get<int32_t>(n1 + 1);
    if (n1 > 0) {
        split_kernel<<<G(n1), 256, 0, st>>>(u1, n1, nullptr, r1y);
        JP_CHECK_LAUNCH();
    }
    int32_t* yval = nullptr;
    const int64_t ny = make_dict(r1y, n1, &yval, ws, st, hist_host);
    uint32_t* flag = ws.get<uint32_t>(n1 + 1);
    uint32_t* gid = ws.get<uint32_t>(n1 + 1);
    uint32_t* d_nx1 = ws.get<uint32_t>(1);
    if (n1 > 0) {
        run_start_kernel<<<G(n1), 256, 0, st>>>(u1, n1, 32, flag);
        JP_CHECK_LAUNCH();
    }
    scan_u32(flag, gid, n1, d_nx1, ws, st);
    const int64_t nx1 = read1(d_nx1, st);
    int32_t* x1val = ws.get<int32_t>(nx1 + 1);
    int32_t* r1off = ws.get<int32_t>(nx1 + 2);
    int32_t* r1ycol = ws.get<int32_t>(n1 + 1);
    int32_t* deg1x = ws.get<int32_t>(nx1 + 1);
    int32_t* deg1y = ws.get<int32_t>(ny + 1);
    JP_CUDA_TRY(cudaMemsetAsync(deg1y, 0, (ny + 1) * sizeof(int32_t), st));
    if (n1 > 0) {
        x_runs_kernel<<<G(n1), 256, 0, st>>>(u1, n1, gid, x1val, r1off);
        JP_CHECK_LAUNCH();
        set_last_kernel<<<1, 1, 0, st>>>(r1off, d_nx1, (int32_t)n1);
        JP_CHECK_LAUNCH();
        lookup_kernel<<<G(n1), 256, 0, st>>>(yval, ny, r1y, n1, r1ycol);
        JP_CHECK_LAUNCH();
        deg_off_kernel<<<G(nx1), 256, 0, st>>>(r1off, nx1, deg1x);
        JP_CHECK_LAUNCH();
        hist_kernel<<<G(n1), 256, 0, st>>>(r1ycol, n1, deg1y);
        JP_CHECK_LAUNCH();
    }
    // ---- R2, R3 indexed by y over R1's y values
    ByY r2, r3;
    index_by_y(&rels[1], yval, ny, r2, ws, st, hist_host);
    index_by_y(&rels[2], yval, ny, r3, ws, st, hist_host);
    so.n_rel[0] = n1;
    so.n_rel[1] = r2.n;
    so.n_rel[2] = r3.n;
    so.nx[0] = nx1;
    so.nx[1] = r2.nx;
    so.nx[2] = r3.nx;
    so.ny = ny;

    // ---- full star join size (an upper bound of OUT)
    unsigned long long* acc = ws.get<unsigned long long>(1);
    JP_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(unsigned long long), st));
    if (ny > 0) {
        star_join_kernel<<<G(ny), 256, 0, st>>>(deg1y, r2.degy, r3.degy, ny, acc);
        JP_CHECK_LAUNCH();
    }
    so.out_join = (double)read1(acc, st);

    // ---- thresholds
    const int64_t N = std::max<int64_t>(std::max<int64_t>(n1, std::max(r2.n, r3.n)), 1);
    if (mode == JP_FIXED) {
        so.d1 = std::min<int64_t>(std::max<int64_t>(fd1, 1), N);
        so.d2 = std::min<int64_t>(std::max<int64_t>(fd2, 1), N);
    } else {
        star_thresholds(N, std::max(so.out_join, 1.0), 3, &so.d1, &so.d2);
    }

    // ---- triples (a1, a2, b), then groups (a1, a2)
    const int sh2 = bits_for(ny);
    const int b2 = bits_for(r2.nx);
    const int sh1 = sh2 + b2;
    if (sh1 + bits_for(nx1) > 64)
        throw Error{JP_EUNSUPPORTED, "x1, x2 and y ids do not fit one 64-bit key"};
    int64_t* tcnt = ws.get<int64_t>(n1 + 1);
    int64_t* toff = ws.get<int64_t>(n1 + 1);
    int64_t* d_T = ws.get<int64_t>(1);
    if (n1 > 0) {
        triple_count_kernel<<<G(n1), 256, 0, st>>>(r1ycol, n1, r2.degy, r3.degy, tcnt);
        JP_CHECK_LAUNCH();
    }
    scan_i64(tcnt, toff, n1, d_T, ws, st);
    const int64_t T = read1(d_T, st);
    if (T >= ((int64_t)1 << 31))
        throw Error{JP_EUNSUPPORTED, "more than 2^31 (x1, x2, y) witness triples"};
    so.triples = T;
    uint64_t* t0 = ws.get<uint64_t>(T > 0 ? T : 1);
    uint64_t* t1 = ws.get<uint64_t>(T > 0 ? T : 1);
    if (T > 0) {
        triple_fill_kernel<<<grid_for(nx1 * 32, 256, 152 * 16), 256, 0, st>>>(
            nx1, r1off, r1ycol, toff, r2.off, r2.col, r3.degy, sh1, sh2, t0);
        JP_CHECK_LAUNCH();
    }
    uint64_t* ts = radix_sort_u64(t0, t1, T, ws, st, hist_host);
    uint32_t* tflag = ws.get<uint32_t>(T + 1);
    uint32_t* tgid = ws.get<uint32_t>(T + 1);
    uint32_t* d_ng = ws.get<uint32_t>(1);
    if (T > 0) {
        run_start_kernel<<<G(T), 256, 0, st>>>(ts, T, sh2, tflag);
        JP_CHECK_LAUNCH();
    }
    scan_u32(tflag, tgid, T, d_ng, ws, st);
    const int64_t ng = read1(d_ng, st);
    so.groups = ng;

    Graph& gv = so.g;
    gv.self = false;
    gv.nx = ng;
    gv.ny = ny;
    gv.nz = r3.nx;
    gv.nr = T;
    gv.ns = r3.n;
    gv.rxoff = ws.get<int32_t>(ng + 2);
    gv.rycol = ws.get<int32_t>(T + 1);
    gv.syoff = r3.off;
    gv.szcol = r3.col;
    gv.deg_sy = r3.degy;
    gv.zval = r3.xval;
    int32_t* ga1 = ws.get<int32_t>(ng + 1);
    int32_t* ga2 = ws.get<int32_t>(ng + 1);
    if (T > 0) {
        group_emit_kernel<<<G(T), 256, 0, st>>>(ts, T, tgid, sh1, sh2, ((uint64_t)1 << b2) - 1,
                                               ((uint64_t)1 << sh2) - 1, ga1, ga2, gv.rxoff,
                                               gv.rycol);
        JP_CHECK_LAUNCH();
    }
    set_last_kernel<<<1, 1, 0, st>>>(gv.rxoff, d_ng, (int32_t)T);
    JP_CHECK_LAUNCH();

    // ---- partition (Section 3.2)
    Partition& p = so.p;
    p.d1 = so.d1;
    p.d2 = so.d2;
    int32_t* pd = ws.get<int32_t>(ng + 1);
    if (ng > 0) {
        pair_heavy_kernel<<<G(ng), 256, 0, st>>>(ga1, ga2, ng, deg1x, r2.degx, so.d2, pd);
        JP_CHECK_LAUNCH();
    }
    p.hx = ws.get<int32_t>(ng + 1);
    p.hx_inv = ws.get<int32_t>(ng + 1);
    p.u = heavy_ids(pd, nullptr, ng, 0, p.hx, p.hx_inv, ws, st);
    int32_t* yc = ws.get<int32_t>(ny + 1);
    if (ny > 0) {
        y_heavy_count_kernel<<<G(ny), 256, 0, st>>>(deg1y, r2.degy, r3.degy, ny, so.d1, yc);
        JP_CHECK_LAUNCH();
    }
    p.hy = ws.get<int32_t>(ny + 1);
    p.hy_inv = ws.get<int32_t>(ny + 1);
    p.v = heavy_ids(yc, nullptr, ny, 1, p.hy, p.hy_inv, ws, st);
    p.hz = ws.get<int32_t>(r3.nx + 1);
    p.hz_inv = ws.get<int32_t>(r3.nx + 1);
    p.w = heavy_ids(r3.degx, nullptr, r3.nx, so.d2, p.hz, p.hz_inv, ws, st);
    build_light_z_lists(r3.off, r3.col, p, ws, st);

    // ---- per-group output values
    so.row1 = ws.get<int32_t>(ng + 1);
    so.row2 = ws.get<int32_t>(ng + 1);
    if (ng > 0) {
        gather_vals_kernel<<<G(ng), 256, 0, st>>>(ga1, ng, x1val, so.row1);
        JP_CHECK_LAUNCH();
        gather_vals_kernel<<<G(ng), 256, 0, st>>>(ga2, ng, r2.xval, so.row2);
        JP_CHECK_LAUNCH();
    }
    (void)d_status;
}

// The star's tail grouped on y: one tuple (g, b) per (a_p, a_q, b) with
// (a_p, b) in P and (a_q, b) in Q, g numbering the distinct pairs (a_p, a_q) in
// value order (so that tuples of g compare as the pairs do); gp[g], gq[g] hold
// the pair's values.  Q*_k with k > 3 is Q*_3 over R1, R2 and the tail
// R3..Rk grouped this way from the right (Section 3.2 groups the star's
// variables the same way for its product).
void pair_relation(const jp_rel* P, const jp_rel* Q, PairRel& out, Arena& ws, cudaStream_t st,
                   uint32_t* hist_host) {
    int32_t* yval = nullptr;
    const int64_t ny = make_dict(P->y, P->n, &yval, ws, st, hist_host);
    ByY bp, bq;
    index_by_y(P, yval, ny, bp, ws, st, hist_host);
    index_by_y(Q, yval, ny, bq, ws, st, hist_host);
    int64_t* cnt = ws.get<int64_t>(ny + 1);
    int64_t* toff = ws.get<int64_t>(ny + 1);
    int64_t* d_tot = ws.get<int64_t>(1);
    if (ny > 0) {
        pair_count_kernel<<<G(ny), 256, 0, st>>>(bp.degy, bq.degy, ny, cnt);
        JP_CHECK_LAUNCH();
    }
    scan_i64(cnt, toff, ny, d_tot, ws, st);
    const int64_t n = ny > 0 ? read1(d_tot, st) : 0;
    if (n >= ((int64_t)1 << 31))
        throw Error{JP_EUNSUPPORTED, "a grouped star tail would hold 2^31 or more tuples"};
    const int shq = bits_for(ny), shp = shq + bits_for(bq.nx);
    if (shp + bits_for(bp.nx) > 64)
        throw Error{JP_EUNSUPPORTED, "grouped star tail keys need more than 64 bits"};
    out.n = n;
    out.x = ws.get<int32_t>(n + 1);
    out.y = ws.get<int32_t>(n + 1);
    out.ng = 0;
    if (n == 0) {
        out.gp = ws.get<int32_t>(1);
        out.gq = ws.get<int32_t>(1);
        return;
    }
    uint64_t* k0 = ws.get<uint64_t>(n);
    uint64_t* k1 = ws.get<uint64_t>(n);
    pair_fill_kernel<<<grid_for(ny * 32, 256, 152 * 16), 256, 0, st>>>(
        ny, bp.off, bp.col, bq.off, bq.col, toff, shp, shq, k0);
    JP_CHECK_LAUNCH();
    uint64_t* ks = radix_sort_u64(k0, k1, n, ws, st, hist_host);
    uint32_t* flag = ws.get<uint32_t>(n);
    uint32_t* gid = ws.get<uint32_t>(n);
    uint32_t* d_ng = ws.get<uint32_t>(1);
    run_start_kernel<<<G(n), 256, 0, st>>>(ks, n, shq, flag);
    JP_CHECK_LAUNCH();
    scan_u32(flag, gid, n, d_ng, ws, st);
    out.ng = read1(d_ng, st);
    out.gp = ws.get<int32_t>(out.ng + 1);
    out.gq = ws.get<int32_t>(out.ng + 1);
    pair_emit_kernel<<<G(n), 256, 0, st>>>(ks, n, gid, shp, shq, ((uint64_t)1 << (shp - shq)) - 1,
                                           ((uint64_t)1 << shq) - 1, bp.xval, bq.xval, yval,
                                           out.x, out.y, out.gp, out.gq);
    JP_CHECK_LAUNCH();
}

namespace {
// columns 2.. of a star result from the grouped third column: follow the
// chain of pair tables (gp: the level's value, gq: the next level's group id,
// or the last relation's value at the last level)
__global__ void expand_kernel(const int32_t* g3, int64_t n, StarChain chain, int32_t* const* cols) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n;
         o += (int64_t)gridDim.x * blockDim.x) {
        int32_t g = g3[o];
        for (int l = 0; l < chain.levels; ++l) {
            cols[l][o] = chain.gp[l][g];
            g = chain.gq[l][g];
        }
        cols[chain.levels][o] = g;
    }
}
}  // namespace

void star_expand(const int32_t* g3, int64_t n, const StarChain& chain, int32_t* const* cols_dev,
                 cudaStream_t st) {
    if (n <= 0) return;
    expand_kernel<<<G(n), 256, 0, st>>>(g3, n, chain, cols_dev);
    JP_CHECK_LAUNCH();
}

}  // namespace jp
