// Witness counts of the two-path query and the set similarity join.
//
// For a pair (a, c) the number of y with R(a, y) and S(c, y) is the entry
// M_ac of the product M1 x M2 (Section 2.2).  The set similarity join
// (Section 1, "Set Similarity") keeps the pairs with M_ac >= c_min; its
// ordered form (Section 4, "Ordered SSJ") lists them by decreasing M_ac.
//
// Algorithm 1's split divides the witnesses disjointly: (a, y, c) is in the
// heavy product iff a, y and c are all heavy (both tuples in R+ and S+);
// otherwise it is one light candidate of a -- taken from S[y] when (a, y) is
// light, from the light z of S[y] when (a, y) is heavy.  Hence
// M_ac = P_ac + L_ac, P the heavy product's entry (0 off the heavy block) and
// L_ac the multiplicity of c among a's light candidates.
//
// x ids are processed in ranges whose candidates fit a budget.  A range's
// candidates are written as keys (x - x0, z id), sorted and run-length
// counted; its rows of P are compacted to the same keys (already in order)
// and merged in, equal keys summed; pairs counted at least c_min are written
// out.  Ranges follow each other in x order, so their concatenation is in
// (x, z) order.
#include <algorithm>
#include <vector>

#include "jp_internal.cuh"

namespace jp {
namespace {

inline int G(int64_t n) { return grid_for(n, 256, 152 * 16); }
inline int GW(int64_t n) { return grid_for(n * 32, 256, 152 * 16); }   // a warp per item

// per entry k = (x, y) of R: the length of the list its candidates come from -- S[y], or
// the light z of S[y] when (x, y) is heavy -- and its x; a warp per x
__global__ void entry_count_kernel(const int32_t* __restrict__ rxoff, const int32_t* __restrict__ rycol,
                                   int64_t nx, const int32_t* __restrict__ hx,
                                   const int32_t* __restrict__ hy, const int32_t* __restrict__ syoff,
                                   const int32_t* __restrict__ sloff,
                                   const int32_t* __restrict__ deg_rx, uint32_t c_min,
                                   int64_t* __restrict__ ecnt, int32_t* __restrict__ rowx) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < nx; x += nw) {
        const bool ah = hx[x] >= 0;
        const bool small = (uint32_t)deg_rx[x] < c_min;   // no pair of x reaches c_min
        for (int32_t k = rxoff[x] + lane; k < rxoff[x + 1]; k += 32) {
            const int32_t b = rycol[k];
            const int32_t j = ah ? hy[b] : -1;
            ecnt[k] = small ? 0 : (j >= 0) ? (sloff[j + 1] - sloff[j]) : (syoff[b + 1] - syoff[b]);
            rowx[k] = (int32_t)x;
        }
    }
}

// The lists col[off[r] .. off[r + 1]) restricted to the values v with deg[v] >= c_min (a pair
// with a smaller set cannot share c_min values): flags, then positions, list and offsets.
__global__ void size_flag_kernel(const int32_t* __restrict__ col, int64_t n,
                                 const int32_t* __restrict__ deg, uint32_t c_min,
                                 uint32_t* __restrict__ flag) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        flag[e] = (uint32_t)deg[col[e]] >= c_min ? 1u : 0u;
}

__global__ void size_compact_kernel(const int32_t* __restrict__ col, int64_t n,
                                    const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                                    int32_t* __restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        if (flag[e]) out[pos[e]] = col[e];
}

__global__ void size_offsets_kernel(const int32_t* __restrict__ off, int64_t rows,
                                    const uint32_t* __restrict__ pos, int32_t* __restrict__ out) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= rows;
         r += (int64_t)gridDim.x * blockDim.x)
        out[r] = (int32_t)pos[off[r]];
}

// coff[x] = offset of x's first candidate (eoff at its first entry)
__global__ void row_offsets_kernel(const int32_t* __restrict__ rxoff, int64_t nx,
                                   const int64_t* __restrict__ eoff, int64_t* __restrict__ coff) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= nx;
         x += (int64_t)gridDim.x * blockDim.x)
        coff[x] = eoff[rxoff[x]];
}

// the candidates of the entries [k0, k1) (the x range [x0, x1)) as keys (x - x0) << 32 | z,
// entry k's at eoff[k] - eoff[k0]; a warp per entry, lanes over its list
__global__ void cand_fill_kernel(int64_t k0, int64_t k1, int64_t x0, const int64_t* __restrict__ eoff,
                                 const int32_t* __restrict__ rowx, const int32_t* __restrict__ rycol,
                                 const int32_t* __restrict__ hx, const int32_t* __restrict__ hy,
                                 const int32_t* __restrict__ syoff, const int32_t* __restrict__ szcol,
                                 const int32_t* __restrict__ sloff, const int32_t* __restrict__ slcol,
                                 const int32_t* __restrict__ deg_rx, uint32_t c_min,
                                 uint64_t* __restrict__ keys) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t c0 = eoff[k0];
    for (int64_t k = k0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); k < k1; k += nw) {
        const int32_t x = rowx[k];
        if ((uint32_t)deg_rx[x] < c_min) continue;
        const int32_t b = rycol[k];
        const int32_t j = hx[x] >= 0 ? hy[b] : -1;
        const int32_t* list;
        int32_t len;
        if (j >= 0) {
            list = slcol + sloff[j];
            len = sloff[j + 1] - sloff[j];
        } else {
            list = szcol + syoff[b];
            len = syoff[b + 1] - syoff[b];
        }
        uint64_t* dst = keys + (eoff[k] - c0);
        const uint64_t hi = (uint64_t)(x - x0) << 32;
        for (int32_t e = lane; e < len; e += 32) dst[e] = hi | (uint32_t)list[e];
    }
}

__global__ void run_mark_kernel(const uint64_t* __restrict__ k, int64_t n, uint32_t* __restrict__ flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || k[i] != k[i - 1]) ? 1u : 0u;
}

__global__ void run_start_kernel(const uint64_t* __restrict__ k, int64_t n,
                                 const uint32_t* __restrict__ flag, const uint32_t* __restrict__ idx,
                                 uint64_t* __restrict__ uk, uint32_t* __restrict__ start) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) {
            uk[idx[i]] = k[i];
            start[idx[i]] = (uint32_t)i;
        }
}

// nonzero entries of the heavy rows [h0, h1) of the count matrix (added to *nonzero) and,
// per row, those of at least c_min; a warp per row
__global__ void heavy_nnz_kernel(const uint32_t* __restrict__ C, int64_t ldc, int64_t h0, int64_t h1,
                                 int64_t w, uint32_t c_min, uint32_t* __restrict__ keep,
                                 unsigned long long* __restrict__ nonzero) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t h = h0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); h < h1; h += nw) {
        const uint32_t* row = C + h * ldc;
        uint32_t s = 0, z = 0;
        for (int64_t j = lane; j < w; j += 32) {
            const uint32_t v = row[j];
            s += v >= c_min;
            z += v != 0u;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_down_sync(0xffffffffu, s, o);
            z += __shfl_down_sync(0xffffffffu, z, o);
        }
        if (lane == 0) {
            keep[h - h0] = s;
            if (z) atomicAdd(nonzero, (unsigned long long)z);
        }
    }
}

// the entries of at least c_min (c_min >= 1) of the heavy rows [h0, h1) as keys
// (x - x0) << 32 | z and counts, row after row, at off[h - h0]
__global__ void heavy_keys_kernel(const uint32_t* __restrict__ C, int64_t ldc, int64_t h0, int64_t h1,
                                  int64_t w, uint32_t c_min, const int32_t* __restrict__ hx_inv,
                                  const int32_t* __restrict__ hz_inv, int64_t x0,
                                  const uint32_t* __restrict__ off, uint64_t* __restrict__ keys,
                                  uint32_t* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t h = h0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); h < h1; h += nw) {
        const uint32_t* row = C + h * ldc;
        const uint64_t hi = (uint64_t)(hx_inv[h] - x0) << 32;
        uint32_t base = off[h - h0];
        for (int64_t j0 = 0; j0 < w; j0 += 32) {
            const int64_t j = j0 + lane;
            const uint32_t v = j < w ? row[j] : 0u;
            const bool kept = v >= c_min && v != 0u;
            const unsigned m = __ballot_sync(0xffffffffu, kept);
            if (kept) {
                const uint32_t p = base + __popc(m & ((1u << lane) - 1u));
                keys[p] = hi | (uint32_t)hz_inv[j];
                cnt[p] = v;
            }
            base += __popc(m);
        }
    }
}

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t* a, int64_t n, uint64_t k) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < k) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// The count of light pair j (the run length of its key among the sorted candidates) plus,
// for x and z heavy, the heavy product's entry, which is then cleared: the entries left in
// the count matrix are the pairs with heavy witnesses only.  Keys are distinct, so each entry
// is read by at most one thread.  keep[j] = count >= c_min.
__global__ void light_count_kernel(const uint64_t* __restrict__ uk, const uint32_t* __restrict__ start,
                                   int64_t m, int64_t nc, int64_t x0, const int32_t* __restrict__ hx,
                                   const int32_t* __restrict__ hz, uint32_t* __restrict__ C,
                                   int64_t ldc, uint32_t c_min, uint32_t* __restrict__ lc,
                                   uint32_t* __restrict__ keep,
                                   unsigned long long* __restrict__ absorbed) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c = (i + 1 < m ? start[i + 1] : (uint32_t)nc) - start[i];
        bool took = false;
        if (C) {
            const uint64_t k = uk[i];
            const int32_t h = hx[x0 + (int64_t)(k >> 32)];
            if (h >= 0) {
                const int32_t zc = hz[(uint32_t)k];
                if (zc >= 0) {
                    uint32_t* e = C + (int64_t)h * ldc + zc;
                    const uint32_t v = *e;
                    if (v != 0u) {
                        c += v;
                        *e = 0u;
                        took = true;
                    }
                }
            }
        }
        lc[i] = c;
        keep[i] = c >= c_min ? 1u : 0u;
        const unsigned b = __ballot_sync(__activemask(), took);
        if (took && (threadIdx.x & 31) == __ffs(b) - 1) atomicAdd(absorbed, (unsigned long long)__popc(b));
    }
}

// first index of row r (keys (r << 32) | z, sorted) for r = 0..rows
__global__ void row_bounds_kernel(const uint64_t* __restrict__ k, int64_t n, int64_t rows,
                                  int64_t* __restrict__ bound) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= rows;
         r += (int64_t)gridDim.x * blockDim.x)
        bound[r] = lower_bound_u64(k, n, (uint64_t)r << 32);
}

// Output of the kept light pairs: pair i goes to (kept light pairs before it, pos[i]) +
// (heavy-only pairs below its key, counted within its row of the heavy list; none when nh = 0)
__global__ void out_light_kernel(const uint64_t* __restrict__ uk, const uint32_t* __restrict__ lc,
                                 const uint32_t* __restrict__ keep, const uint32_t* __restrict__ pos,
                                 int64_t m, const uint64_t* __restrict__ hk,
                                 const int64_t* __restrict__ hrow, int64_t x0,
                                 const int32_t* __restrict__ xval, const int32_t* __restrict__ zval,
                                 int32_t* __restrict__ ox, int32_t* __restrict__ oz,
                                 int32_t* __restrict__ oc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[i]) continue;
        const uint64_t key = uk[i];
        const int64_t r = (int64_t)(key >> 32);
        int64_t p = pos[i];
        if (hrow) {
            const int64_t s0 = hrow[r];
            p += s0 + lower_bound_u64(hk + s0, hrow[r + 1] - s0, key);
        }
        ox[p] = xval[x0 + r];
        oz[p] = zval[(uint32_t)key];
        oc[p] = (int32_t)lc[i];
    }
}

// Output of the heavy-only pairs (all kept): pair i goes to i + (kept light pairs below its
// key: pos at its insertion point in the light list, found within its row)
__global__ void out_heavy_kernel(const uint64_t* __restrict__ hk, const uint32_t* __restrict__ hc,
                                 int64_t nh, const uint64_t* __restrict__ uk,
                                 const int64_t* __restrict__ lrow, const uint32_t* __restrict__ pos,
                                 int64_t x0, const int32_t* __restrict__ xval,
                                 const int32_t* __restrict__ zval, int32_t* __restrict__ ox,
                                 int32_t* __restrict__ oz, int32_t* __restrict__ oc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nh;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = hk[i];
        const int64_t r = (int64_t)(key >> 32);
        const int64_t s0 = lrow[r];
        const int64_t q = s0 + lower_bound_u64(uk + s0, lrow[r + 1] - s0, key);
        const int64_t p = i + pos[q];
        ox[p] = xval[x0 + r];
        oz[p] = zval[(uint32_t)key];
        oc[p] = (int32_t)hc[i];
    }
}

// sort keys for decreasing count, ties in position order: (~count) << 32 | position
__global__ void count_order_keys_kernel(const int32_t* __restrict__ c, int64_t n,
                                        uint64_t* __restrict__ k) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        k[i] = ((uint64_t)(~(uint32_t)c[i]) << 32) | (uint32_t)i;
}

__global__ void gather3_kernel(const uint64_t* __restrict__ k, int64_t n, const int32_t* __restrict__ x,
                               const int32_t* __restrict__ z, const int32_t* __restrict__ c,
                               int32_t* __restrict__ ox, int32_t* __restrict__ oz,
                               int32_t* __restrict__ oc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = (uint32_t)k[i];
        ox[i] = x[j];
        oz[i] = z[j];
        oc[i] = c[j];
    }
}

template <class T> T read1(const T* d, cudaStream_t st) {
    T v{};
    JP_CUDA_TRY(cudaMemcpyAsync(&v, d, sizeof(T), cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaStreamSynchronize(st));
    return v;
}

// Scratch that grows on demand (the arena never frees within a query).
template <class T> struct Grow {
    T* p = nullptr;
    int64_t cap = -1;
    T* need(int64_t n, Arena& ws) {
        if (n > cap) {
            cap = std::max<int64_t>(n, 1);
            p = ws.get<T>((size_t)cap);
        }
        return p;
    }
};

}  // namespace

void count_pairs(const Graph& g, const Partition& p, const Heavy& h, int64_t c_min, int order,
                 CountResult& out, Arena& ws, cudaStream_t st, uint32_t* d_status,
                 uint32_t* hist_host, int64_t chunk_candidates) {
    out = CountResult{};
    const int64_t nx = g.nx;
    if (nx == 0) return;
    if (c_min < 1) c_min = 1;
    const uint32_t cmin = c_min > 0x7fffffff ? 0x7fffffffu : (uint32_t)c_min;

    // heavy product entries
    uint32_t* C = nullptr;
    if (h.present) {
        // an entry counts heavy y shared by a pair, at most v; the FP32
        // accumulators hold every integer exactly only below 2^24
        if (p.v >= ((int64_t)1 << 24))
            throw Error{JP_EUNSUPPORTED, "2^24 or more heavy y: product counts would be inexact"};
        const size_t bytes = (size_t)h.u_pad * (size_t)h.w_pad * sizeof(uint32_t);
        if (bytes > ((size_t)1 << 36))
            throw Error{JP_EUNSUPPORTED, "the heavy count matrix would exceed 64 GiB"};
        C = ws.get<uint32_t>((size_t)h.u_pad * (size_t)h.w_pad);
        heavy_gemm_counts(h, C, d_status, st);
    }

    // with c_min > 1, S's lists (and the light-z lists of heavy y) keep only the z whose set
    // has at least c_min values, and x with fewer than c_min values have no candidates
    const int32_t* syoff = g.syoff;
    const int32_t* szcol = g.szcol;
    const int32_t* sloff = p.sloff;
    const int32_t* slcol = p.slcol;
    auto restrict_lists = [&](const int32_t* off, const int32_t* col, int64_t rows, int64_t n,
                              const int32_t** off_out, const int32_t** col_out) {
        uint32_t* flag = ws.get<uint32_t>(n + 1);
        uint32_t* pos = ws.get<uint32_t>(n + 1);
        int32_t* c2 = ws.get<int32_t>(n + 1);
        int32_t* o2 = ws.get<int32_t>(rows + 1);
        if (n > 0) {
            size_flag_kernel<<<G(n), 256, 0, st>>>(col, n, g.deg_sz, cmin, flag);
            JP_CHECK_LAUNCH();
        }
        scan_u32(flag, pos, n, pos + n, ws, st);
        if (n > 0) {
            size_compact_kernel<<<G(n), 256, 0, st>>>(col, n, flag, pos, c2);
            JP_CHECK_LAUNCH();
        }
        size_offsets_kernel<<<G(rows + 1), 256, 0, st>>>(off, rows, pos, o2);
        JP_CHECK_LAUNCH();
        *off_out = o2;
        *col_out = c2;
    };
    if (cmin > 1) {
        restrict_lists(g.syoff, g.szcol, g.ny, g.ns, &syoff, &szcol);
        if (p.v > 0) {
            int32_t nl = 0;
            JP_CUDA_TRY(cudaMemcpyAsync(&nl, p.sloff + p.v, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            JP_CUDA_TRY(cudaStreamSynchronize(st));
            restrict_lists(p.sloff, p.slcol, p.v, nl, &sloff, &slcol);
        }
    }

    // light candidates per entry of R, their offsets, and per x
    const int64_t nr = g.nr;
    int64_t* ecnt = ws.get<int64_t>(nr + 1);
    int64_t* eoff = ws.get<int64_t>(nr + 1);
    int32_t* rowx = ws.get<int32_t>(nr + 1);
    int64_t* coff = ws.get<int64_t>(nx + 1);
    entry_count_kernel<<<GW(nx), 256, 0, st>>>(g.rxoff, g.rycol, nx, p.hx, p.hy, syoff, sloff,
                                               g.deg_rx, cmin, ecnt, rowx);
    JP_CHECK_LAUNCH();
    scan_i64(ecnt, eoff, nr, eoff + nr, ws, st);
    row_offsets_kernel<<<G(nx + 1), 256, 0, st>>>(g.rxoff, nx, eoff, coff);
    JP_CHECK_LAUNCH();
    std::vector<int64_t> hoff_host((size_t)nx + 1);
    std::vector<int32_t> rxoff_host((size_t)nx + 1);
    JP_CUDA_TRY(cudaMemcpyAsync(hoff_host.data(), coff, (nx + 1) * sizeof(int64_t),
                                cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaMemcpyAsync(rxoff_host.data(), g.rxoff, (nx + 1) * sizeof(int32_t),
                                cudaMemcpyDeviceToHost, st));
    std::vector<int32_t> hx_inv_host((size_t)p.u);
    if (p.u > 0)
        JP_CUDA_TRY(cudaMemcpyAsync(hx_inv_host.data(), p.hx_inv, p.u * sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaStreamSynchronize(st));
    out.candidates = hoff_host[nx];
    int64_t max_row = 0;
    for (int64_t x = 0; x < nx; ++x) max_row = std::max(max_row, hoff_host[x + 1] - hoff_host[x]);
    if (max_row >= ((int64_t)1 << 31))
        throw Error{JP_EUNSUPPORTED, "one x has 2^31 or more light candidates"};
    const int64_t cap = std::max<int64_t>(
        std::max<int64_t>(std::min<int64_t>(chunk_candidates, out.candidates), 1), max_row);

    uint64_t* keys = ws.get<uint64_t>(cap);
    uint64_t* tmp = ws.get<uint64_t>(cap);
    uint32_t* flag = ws.get<uint32_t>(cap);
    uint32_t* idx = ws.get<uint32_t>(cap + 1);
    uint64_t* uk = ws.get<uint64_t>(cap);
    uint32_t* start = ws.get<uint32_t>(cap);
    uint32_t* lc = ws.get<uint32_t>(cap);
    uint32_t* d_total = ws.get<uint32_t>(1);
    unsigned long long* d_absorbed = ws.get<unsigned long long>(2);   // absorbed, nonzero
    JP_CUDA_TRY(cudaMemsetAsync(d_absorbed, 0, 2 * sizeof(unsigned long long), st));
    Grow<uint32_t> hkeep, hoffs, hc;
    Grow<uint64_t> hk;
    Grow<int64_t> lrow, hrow;

    struct Piece { int32_t* x; int32_t* z; int32_t* c; int64_t n; };
    std::vector<Piece> pieces;
    int64_t total = 0;
    // device time of the phases of every range: fill | sort and run lengths | counts and output
    struct Events {
        cudaEvent_t e[4] = {};
        Events() { for (auto& x : e) cudaEventCreate(&x); }
        ~Events() { for (auto& x : e) cudaEventDestroy(x); }
    } ev;
    auto elapsed = [](cudaEvent_t a, cudaEvent_t b) {
        float v = 0;
        if (cudaEventElapsedTime(&v, a, b) != cudaSuccess) { cudaGetLastError(); v = 0; }
        return (double)v;
    };
    for (int64_t x0 = 0; x0 < nx;) {
        // the longest range of x from x0 whose candidates fit the scratch
        int64_t x1 = std::upper_bound(hoff_host.begin() + x0 + 1, hoff_host.end(),
                                      hoff_host[x0] + cap) - hoff_host.begin() - 1;
        if (x1 <= x0) x1 = x0 + 1;
        const int64_t nc = hoff_host[x1] - hoff_host[x0];
        const int64_t rows = x1 - x0;
        // light pairs of the range: sorted keys, run starts
        int64_t m = 0;
        JP_CUDA_TRY(cudaEventRecord(ev.e[0], st));
        JP_CUDA_TRY(cudaEventRecord(ev.e[1], st));
        if (nc > 0) {
            const int64_t k0 = rxoff_host[x0], k1 = rxoff_host[x1];
            cand_fill_kernel<<<GW(k1 - k0), 256, 0, st>>>(k0, k1, x0, eoff, rowx, g.rycol, p.hx, p.hy,
                                                          syoff, szcol, sloff, slcol, g.deg_rx, cmin,
                                                          keys);
            JP_CHECK_LAUNCH();
            JP_CUDA_TRY(cudaEventRecord(ev.e[1], st));
            uint64_t* sk = radix_sort_u64(keys, tmp, nc, ws, st, hist_host);
            run_mark_kernel<<<G(nc), 256, 0, st>>>(sk, nc, flag);
            JP_CHECK_LAUNCH();
            scan_u32(flag, idx, nc, d_total, ws, st);
            run_start_kernel<<<G(nc), 256, 0, st>>>(sk, nc, flag, idx, uk, start);
            JP_CHECK_LAUNCH();
            m = read1(d_total, st);
        }
        JP_CUDA_TRY(cudaEventRecord(ev.e[2], st));
        // heavy rows of the range
        const int64_t h0 = std::lower_bound(hx_inv_host.begin(), hx_inv_host.end(), (int32_t)x0) -
                           hx_inv_host.begin();
        const int64_t h1 = std::lower_bound(hx_inv_host.begin(), hx_inv_host.end(),
                                            (int32_t)std::min<int64_t>(x1, 0x7fffffff)) -
                           hx_inv_host.begin();
        const bool heavy_rows = C && h1 > h0;
        // final counts of the light pairs (the product's entries of heavy x and z taken in and
        // cleared), kept flags and their positions (idx[m] = kept light pairs)
        int64_t ml = 0;
        if (m > 0) {
            light_count_kernel<<<G(m), 256, 0, st>>>(uk, start, m, nc, x0, p.hx, p.hz,
                                                     heavy_rows ? C : nullptr, h.w_pad, cmin, lc, flag,
                                                     d_absorbed);
            JP_CHECK_LAUNCH();
            scan_u32(flag, idx, m, idx + m, ws, st);
        } else {
            JP_CUDA_TRY(cudaMemsetAsync(idx, 0, sizeof(uint32_t), st));
        }
        // heavy-only pairs of at least c_min
        int64_t nh = 0;
        if (heavy_rows) {
            uint32_t* kp = hkeep.need(h1 - h0, ws);
            uint32_t* off = hoffs.need(h1 - h0, ws);
            heavy_nnz_kernel<<<GW(h1 - h0), 256, 0, st>>>(C, h.w_pad, h0, h1, p.w, cmin, kp,
                                                          d_absorbed + 1);
            JP_CHECK_LAUNCH();
            scan_u32(kp, off, h1 - h0, d_total, ws, st);
            nh = read1(d_total, st);
            if (nh > 0) {
                heavy_keys_kernel<<<GW(h1 - h0), 256, 0, st>>>(C, h.w_pad, h0, h1, p.w, cmin,
                                                               p.hx_inv, p.hz_inv, x0, off,
                                                               hk.need(nh, ws), hc.need(nh, ws));
                JP_CHECK_LAUNCH();
            }
        }
        ml = m > 0 ? read1(idx + m, st) : 0;
        // both lists written to the range's output in key order
        const int64_t nk = ml + nh;
        if (nk > 0) {
            Piece pc{ws.get<int32_t>(nk), ws.get<int32_t>(nk), ws.get<int32_t>(nk), nk};
            int64_t* hr = nullptr;
            if (nh > 0) {
                hr = hrow.need(rows + 1, ws);
                row_bounds_kernel<<<G(rows + 1), 256, 0, st>>>(hk.p, nh, rows, hr);
                JP_CHECK_LAUNCH();
            }
            if (ml > 0) {
                out_light_kernel<<<G(m), 256, 0, st>>>(uk, lc, flag, idx, m, hk.p, hr, x0, g.xval,
                                                       g.zval, pc.x, pc.z, pc.c);
                JP_CHECK_LAUNCH();
            }
            if (nh > 0) {
                int64_t* lr = lrow.need(rows + 1, ws);
                row_bounds_kernel<<<G(rows + 1), 256, 0, st>>>(uk, m, rows, lr);
                JP_CHECK_LAUNCH();
                out_heavy_kernel<<<G(nh), 256, 0, st>>>(hk.p, hc.p, nh, uk, lr, idx, x0, g.xval,
                                                        g.zval, pc.x, pc.z, pc.c);
                JP_CHECK_LAUNCH();
            }
            pieces.push_back(pc);
            total += nk;
        }
        out.light_pairs += m;
        JP_CUDA_TRY(cudaEventRecord(ev.e[3], st));
        JP_CUDA_TRY(cudaEventSynchronize(ev.e[3]));
        out.ms_fill += elapsed(ev.e[0], ev.e[1]);
        out.ms_sort += elapsed(ev.e[1], ev.e[2]);
        out.ms_merge += elapsed(ev.e[2], ev.e[3]);
        ++out.ranges;
        x0 = x1;
    }
    {
        unsigned long long hv[2];
        JP_CUDA_TRY(cudaMemcpyAsync(hv, d_absorbed, sizeof(hv), cudaMemcpyDeviceToHost, st));
        JP_CUDA_TRY(cudaStreamSynchronize(st));
        out.heavy_pairs = (int64_t)(hv[0] + hv[1]);   // entries taken by light pairs + the rest
    }
    if (total >= ((int64_t)1 << 32)) throw Error{JP_EUNSUPPORTED, "2^32 or more result pairs"};
    // the pieces one after another
    int32_t* X = ws.get<int32_t>(total + 1);
    int32_t* Z = ws.get<int32_t>(total + 1);
    int32_t* K = ws.get<int32_t>(total + 1);
    int64_t at = 0;
    for (const Piece& pc : pieces) {
        JP_CUDA_TRY(cudaMemcpyAsync(X + at, pc.x, pc.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        JP_CUDA_TRY(cudaMemcpyAsync(Z + at, pc.z, pc.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        JP_CUDA_TRY(cudaMemcpyAsync(K + at, pc.c, pc.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        at += pc.n;
    }
    if (order == 1 && total > 1) {
        uint64_t* ok0 = ws.get<uint64_t>(total);
        uint64_t* ok1 = ws.get<uint64_t>(total);
        count_order_keys_kernel<<<G(total), 256, 0, st>>>(K, total, ok0);
        JP_CHECK_LAUNCH();
        uint64_t* s = radix_sort_u64(ok0, ok1, total, ws, st, hist_host);
        int32_t* X2 = ws.get<int32_t>(total);
        int32_t* Z2 = ws.get<int32_t>(total);
        int32_t* K2 = ws.get<int32_t>(total);
        gather3_kernel<<<G(total), 256, 0, st>>>(s, total, X, Z, K, X2, Z2, K2);
        JP_CHECK_LAUNCH();
        X = X2;
        Z = Z2;
        K = K2;
    }
    out.x = X;
    out.z = Z;
    out.cnt = K;
    out.n = total;
}

}  // namespace jp
