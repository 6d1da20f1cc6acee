// Threshold selection (Section 3.1 closed forms, Section 5 cost-based
// optimizer, Algorithm 3).
//
// The degree indexes of Section 5 are built on the device as exact degree
// histograms: values with degree <= HMAX are counted per degree, the few with
// larger degree are listed individually.  The host then answers every index
// query of Algorithm 3 exactly:
//   sum(y_d)   = sum over light y (deg <= d) of deg_R(y) * deg_S(y)
//                (the light-y join size; deg^2 for a self-join)
//   sum(x_d)   = sum over light x of sum_{b in R[x]} deg_S(b)
//                (the deduplication effort of light x)
//   cdfx(y_d)  = sum over light y of deg_R(y)
//   count(w_d) = number of values of w with degree <= d
// The y degree used for y is max(deg_R(y), deg_S(y)) (the partition rule).
#include <algorithm>
#include <cmath>

#include "jp_internal.cuh"

namespace jp {
namespace {

constexpr int HMAX = 4096;

struct DevHist {
    unsigned long long x_cnt[HMAX + 1];
    unsigned long long x_cand[HMAX + 1];
    unsigned long long y_cnt[HMAX + 1];
    unsigned long long y_w[HMAX + 1];
    unsigned long long y_r[HMAX + 1];
    unsigned long long z_cnt[HMAX + 1];
    unsigned int n_xo, n_yo, n_zo;
};

struct Over { long long deg; unsigned long long a, b; };

// Degrees below SB are counted per block in shared memory and added to the
// global bins once per block (most values have small degrees, so global
// atomics on a few bins would serialise).
constexpr int SB = 1024;

// x bins: count and candidates (xsum: each x's join candidates, from the build)
__global__ void hist_x_kernel(int64_t nx, const int32_t* __restrict__ rxoff,
                              const int64_t* __restrict__ xsum, DevHist* H, Over* xo) {
    __shared__ unsigned long long s_cnt[SB], s_cand[SB];
    for (int i = threadIdx.x; i < SB; i += blockDim.x) s_cnt[i] = s_cand[i] = 0;
    __syncthreads();
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nx;
         a += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = rxoff[a + 1] - rxoff[a];
        const unsigned long long c = (unsigned long long)xsum[a];
        if (d < SB) {
            atomicAdd(&s_cnt[d], 1ull);
            atomicAdd(&s_cand[d], c);
        } else if (d <= HMAX) {
            atomicAdd(&H->x_cnt[d], 1ull);
            atomicAdd(&H->x_cand[d], c);
        } else {
            const unsigned int i = atomicAdd(&H->n_xo, 1u);
            xo[i] = Over{d, c, 0};
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SB; i += blockDim.x)
        if (s_cnt[i]) {
            atomicAdd(&H->x_cnt[i], s_cnt[i]);
            atomicAdd(&H->x_cand[i], s_cand[i]);
        }
}

__global__ void hist_y_kernel(int64_t ny, const int32_t* deg_ry, const int32_t* deg_sy,
                              DevHist* H, Over* yo) {
    __shared__ unsigned long long s_cnt[SB], s_w[SB], s_r[SB];
    for (int i = threadIdx.x; i < SB; i += blockDim.x) s_cnt[i] = s_w[i] = s_r[i] = 0;
    __syncthreads();
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < ny;
         b += (int64_t)gridDim.x * blockDim.x) {
        const long long r = deg_ry[b], s = deg_sy[b];
        const long long d = r > s ? r : s;
        const unsigned long long wgt = (unsigned long long)(r * s);
        if (d < SB) {
            atomicAdd(&s_cnt[d], 1ull);
            atomicAdd(&s_w[d], wgt);
            atomicAdd(&s_r[d], (unsigned long long)r);
        } else if (d <= HMAX) {
            atomicAdd(&H->y_cnt[d], 1ull);
            atomicAdd(&H->y_w[d], wgt);
            atomicAdd(&H->y_r[d], (unsigned long long)r);
        } else {
            const unsigned int i = atomicAdd(&H->n_yo, 1u);
            yo[i] = Over{d, wgt, (unsigned long long)r};
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SB; i += blockDim.x)
        if (s_cnt[i]) {
            atomicAdd(&H->y_cnt[i], s_cnt[i]);
            atomicAdd(&H->y_w[i], s_w[i]);
            atomicAdd(&H->y_r[i], s_r[i]);
        }
}

__global__ void hist_z_kernel(int64_t nz, const int32_t* deg_sz, DevHist* H, Over* zo) {
    __shared__ unsigned long long s_cnt[SB];
    for (int i = threadIdx.x; i < SB; i += blockDim.x) s_cnt[i] = 0;
    __syncthreads();
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nz;
         c += (int64_t)gridDim.x * blockDim.x) {
        const long long d = deg_sz[c];
        if (d < SB) {
            atomicAdd(&s_cnt[d], 1ull);
        } else if (d <= HMAX) {
            atomicAdd(&H->z_cnt[d], 1ull);
        } else {
            const unsigned int i = atomicAdd(&H->n_zo, 1u);
            zo[i] = Over{d, 0, 0};
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SB; i += blockDim.x)
        if (s_cnt[i]) atomicAdd(&H->z_cnt[i], s_cnt[i]);
}

// Cumulative index over degrees: values with degree <= delta.
struct Index {
    std::vector<double> cnt, s1, s2;     // prefix over exact bins 0..HMAX
    std::vector<long long> od;           // overflow degrees, sorted
    std::vector<double> oc, o1, o2;      // prefix over overflow entries
    double total_cnt = 0;

    void build(const unsigned long long* c, const unsigned long long* a,
               const unsigned long long* b, std::vector<Over> over) {
        cnt.assign(HMAX + 2, 0);
        s1.assign(HMAX + 2, 0);
        s2.assign(HMAX + 2, 0);
        for (int d = 0; d <= HMAX; ++d) {
            cnt[d + 1] = cnt[d] + (double)c[d];
            s1[d + 1] = s1[d] + (a ? (double)a[d] : 0.0);
            s2[d + 1] = s2[d] + (b ? (double)b[d] : 0.0);
        }
        std::sort(over.begin(), over.end(), [](const Over& p, const Over& q) { return p.deg < q.deg; });
        od.clear();
        oc.assign(over.size() + 1, 0);
        o1.assign(over.size() + 1, 0);
        o2.assign(over.size() + 1, 0);
        for (size_t i = 0; i < over.size(); ++i) {
            od.push_back(over[i].deg);
            oc[i + 1] = oc[i] + 1;
            o1[i + 1] = o1[i] + (double)over[i].a;
            o2[i + 1] = o2[i] + (double)over[i].b;
        }
        total_cnt = cnt[HMAX + 1] + oc[over.size()];
    }
    // sums over values with degree <= delta; which = 0 count, 1 first, 2 second
    double le(double delta, int which) const {
        const std::vector<double>& P = which == 0 ? cnt : (which == 1 ? s1 : s2);
        const std::vector<double>& O = which == 0 ? oc : (which == 1 ? o1 : o2);
        const long long d = (long long)std::floor(delta);
        if (d < 0) return 0;
        if (d <= HMAX) return P[d + 1];
        size_t k = std::upper_bound(od.begin(), od.end(), d) - od.begin();
        return P[HMAX + 1] + O[k];
    }
    double gt_count(double delta) const { return total_cnt - le(delta, 0); }
};

int64_t clamp_delta(double d, int64_t N) {
    if (!(d >= 1.0)) return 1;
    double f = std::floor(d);
    if (f > (double)N) return N > 0 ? N : 1;
    return (int64_t)f;
}

}  // namespace

// Default calibration constants of the GPU cost model (seconds), in the
// roles of Table 2: T_I per light candidate inserted into a deduplication
// structure, T_m per matrix element / per-x structure set up, T_s per
// sequential step of a scan of the light-y list for every x, and the product
// time model M_hat(u,v,w) = 2uvw / mm_rate + mm_fixed.  They are a
// non-negative least-squares fit (with a free offset per relation) to
// whole-query times measured on GB300 at 49 fixed threshold pairs on each of
// 789 seeded power-law self-joins of 1e5 to 5e6 tuples, over the points
// within 3x of each relation's fastest.  The fit gives T_I = 0: the bitmap
// and merge kernels take an extra candidate almost for free (the light cost
// follows the light-y tuples, the T_s term, and the distinct outputs, which
// the thresholds do not change), so the heavy product pays only where it
// removes many light-y tuples.
jp_cost_model default_cost_model() {
    jp_cost_model K;
    K.T_I = 0.0;
    K.T_m = 1.34e-12;
    K.T_s = 5.04e-16;
    K.mm_rate = 3.85e15;
    K.mm_fixed = 1.46e-4;
    K.eps = 0.05;
    K.wcoj_factor = 20.0;
    K.judge = 3.0;
    return K;
}

bool valid_cost_model(const jp_cost_model& K) {
    auto fin = [](double v) { return std::isfinite(v); };
    return fin(K.T_I) && fin(K.T_m) && fin(K.T_s) && fin(K.mm_rate) && fin(K.mm_fixed) &&
           fin(K.eps) && fin(K.wcoj_factor) && fin(K.judge) && K.T_I >= 0 && K.T_m >= 0 &&
           K.T_s >= 0 && K.mm_rate > 0 && K.mm_fixed >= 0 && K.eps > 0 && K.eps < 1 &&
           K.wcoj_factor >= 0 && K.judge >= 1;
}

double out_estimate(double dom_x, double out_join, double N) {
    if (N <= 0) return 0;
    double lo = std::max(dom_x, (out_join / N) * (out_join / N));
    double hi = std::min(dom_x * dom_x, out_join);
    return std::sqrt(lo * hi);
}

void select_thresholds(const Graph& g, int mode, int64_t fd1, int64_t fd2, int64_t* d1,
                       int64_t* d2, double* out_est, Arena& ws, cudaStream_t st,
                       const jp_cost_model& K, jp_mlp* predictor, int* judged) {
    if (judged) *judged = 0;
    // N: the larger relation after R's dangling tuples are dropped (Section
    // 3.1 assumes |R| = |S| = N)
    const int64_t N = std::max<int64_t>(std::max(g.nr, g.ns), 1);
    *out_est = out_estimate((double)g.nx, g.out_join, (double)N);
    if (mode == JP_FIXED) {
        *d1 = std::min<int64_t>(std::max<int64_t>(fd1, 1), N);
        *d2 = std::min<int64_t>(std::max<int64_t>(fd2, 1), N);
        return;
    }
    if (mode == JP_CLOSED_FORM) {
        const double OUT = std::max(*out_est, 1.0);
        const double n = (double)N;
        double a, b;
        if (OUT <= n) {
            const double c = std::cbrt(OUT);
            a = c;
            b = n / (c * c);
        } else {
            a = b = std::cbrt(2.0 * n * n / (n + OUT));
        }
        *d1 = clamp_delta(a, N);
        *d2 = clamp_delta(b, N);
        return;
    }
    // JP_LEARNED: the model predicts (l1, l2); the cost model below then judges
    // them against its own choice and keeps them unless they cost more than
    // K.judge times as much
    int64_t l1 = 0, l2 = 0;
    if (mode == JP_LEARNED) {
        if (!predictor) throw Error{JP_EINVAL, "JP_LEARNED needs a model (jp_set_predictor)"};
        float f[128];
        graph_features(g, f, ws, st);
        mlp_predict(predictor, f, N, &l1, &l2);
    } else if (mode != JP_COST_MODEL) {
        throw Error{JP_EINVAL, "unknown threshold mode"};
    }
    // ---- Algorithm 3 on exact degree indexes
    if (mode == JP_COST_MODEL && g.out_join <= K.wcoj_factor * (double)N) {  // plain worst-case optimal join
        *d1 = N;
        *d2 = N;
        return;
    }
    DevHist* H = ws.get<DevHist>(1);
    Over* xo = ws.get<Over>(g.nx + 1);
    Over* yo = ws.get<Over>(g.ny + 1);
    Over* zo = ws.get<Over>(g.nz + 1);
    JP_CUDA_TRY(cudaMemsetAsync(H, 0, sizeof(DevHist), st));
    if (g.nx) {
        if (!g.xsum) throw Error{JP_EINVAL, "threshold selection needs the per-x candidate sums"};
        hist_x_kernel<<<grid_for(g.nx, 256, 152 * 4), 256, 0, st>>>(g.nx, g.rxoff, g.xsum, H, xo);
        JP_CHECK_LAUNCH();
    }
    if (g.ny) {
        hist_y_kernel<<<grid_for(g.ny, 256, 152 * 4), 256, 0, st>>>(g.ny, g.deg_ry, g.deg_sy, H, yo);
        JP_CHECK_LAUNCH();
    }
    if (!g.self && g.nz) {
        hist_z_kernel<<<grid_for(g.nz, 256, 152 * 4), 256, 0, st>>>(g.nz, g.deg_sz, H, zo);
        JP_CHECK_LAUNCH();
    }
    std::vector<DevHist> hh(1);
    JP_CUDA_TRY(cudaMemcpyAsync(hh.data(), H, sizeof(DevHist), cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaStreamSynchronize(st));
    const DevHist& h = hh[0];
    std::vector<Over> vx(h.n_xo), vy(h.n_yo), vz(h.n_zo);
    if (h.n_xo) JP_CUDA_TRY(cudaMemcpy(vx.data(), xo, h.n_xo * sizeof(Over), cudaMemcpyDeviceToHost));
    if (h.n_yo) JP_CUDA_TRY(cudaMemcpy(vy.data(), yo, h.n_yo * sizeof(Over), cudaMemcpyDeviceToHost));
    if (h.n_zo) JP_CUDA_TRY(cudaMemcpy(vz.data(), zo, h.n_zo * sizeof(Over), cudaMemcpyDeviceToHost));
    Index IX, IY, IZ;
    IX.build(h.x_cnt, h.x_cand, nullptr, vx);
    IY.build(h.y_cnt, h.y_w, h.y_r, vy);
    if (g.self) IZ = IX; else IZ.build(h.z_cnt, nullptr, nullptr, vz);

    const double OUT = std::max(*out_est, 1.0);
    const double n = (double)N;
    const double dom_x = (double)g.nx;
    auto cost = [&](double a, double b) {
        double light = K.T_I * IY.le(a, 1) + K.T_I * IX.le(b, 1) + K.T_m * dom_x +
                       K.T_s * IY.le(a, 2) * dom_x;
        double u = IX.gt_count(b), v = IY.gt_count(a), w = IZ.gt_count(b);
        double heavy = 0;
        if (u > 0 && v > 0 && w > 0)
            heavy = 2.0 * u * v * w / K.mm_rate + K.mm_fixed + K.T_m * (u * v + u * w);
        return light + heavy;
    };
    double a = n, b = std::max(n * a / OUT, 1.0);
    double prev_cost = INFINITY, pa = a, pb = b;
    const bool wcoj = g.out_join <= K.wcoj_factor * (double)N;
    for (int it = 0; it < 100000 && !wcoj; ++it) {
        double c = cost(a, b);
        if (c > prev_cost) break;
        prev_cost = c;
        pa = a;
        pb = b;
        if (a <= 1.0) break;
        a = std::max(a * (1.0 - K.eps), 1.0);
        b = std::max(n * a / OUT, 1.0);
    }
    if (mode == JP_LEARNED) {
        const double cl = cost((double)l1, (double)l2), ca = cost(pa, pb);
        // the prediction's heavy block: FP8 operands (u x v, w x v bytes) and
        // the product's bit matrix (u x w bits); it must also fit in half of
        // the device memory that is free now
        const double u = IX.gt_count((double)l2), v = IY.gt_count((double)l1),
                     w = IZ.gt_count((double)l2);
        size_t free_b = 0, total_b = 0;
        JP_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
        const bool fits = v * (u + w) + u * w / 8.0 <= 0.5 * (double)free_b;
        if (fits && cl <= K.judge * ca) {
            *d1 = l1;
            *d2 = l2;
            if (judged) *judged = 1;
            return;
        }
        if (judged) *judged = 2;
    }
    *d1 = clamp_delta(pa, N);
    *d2 = clamp_delta(pb, N);
}

}  // namespace jp
