// Light part and union (Algorithm 1, "T <- (R^- join S) union (R join S^-)"
// and "T <- T union {(a,c) : M_ac > 0}"; deduplication as in Section 6).
//
// The light witnesses are enumerated with the disjoint split
// (R^- join S) union (R^+ join S^-), which reaches the same set as the
// paper's two overlapping joins without enumerating R^- join S^- twice:
//   x = a light:  candidates  = union of S[b] over b in R[a]
//   x = a heavy:  candidates  = union of S[b] over light b in R[a]
//                             + union of S^-[b] (light z only) over heavy b
// and every distinct candidate z of a is one output pair (a, z).
//
// Per x the candidate count c(a) is computed first; each x then goes to the
// cheapest deduplication for its size, mirroring the paper's choice between
// a dense marker vector and append-then-sort (Section 6, "Deduplication"):
//   one list      a light x with a single neighbour list is already sorted
//                 and distinct: the output pass copies S[b] in place
//   c <= 256      a warp sorts the candidates in shared memory (bitonic)
//   c <= 8192     (at most 64 lists) a block merges the lists, which are
//                 already sorted, pairwise in shared memory (three buffer
//                 sizes: 2048, 4096 and 8192)
//   c <= 2048     (more than 64 lists) a warp bucket-sorts them over the
//                 row's z range (linear work)
//   larger, and every heavy x: a block marks z in a shared-memory bitmap
//                 over the z domain (windowed when the domain is larger than
//                 shared memory) with a one-bit-per-word summary, so that
//                 emitting and clearing cost grows with the touched words,
//                 not with the domain.  Heavy rows also OR in their row of
//                 the heavy product bitmap G: this is the union with the
//                 matrix part.  Set bits are emitted in z order.
// Each x's sorted distinct list goes to a scratch buffer at an offset taken
// by one atomic add; the output pass then places the lists in x order.  The
// sort and merge classes read the lists of S as z values (szval, in id
// order, which is value order) and write values; the bitmap class marks and
// writes z ids, which the output pass maps to values.
#include "jp_internal.cuh"

namespace jp {
namespace {

constexpr int32_t KEY_PAD = 0x7fffffff;
constexpr int W_CAP = 256;            // small warp class capacity
constexpr int W2_CAP = 2048;          // warp bucket class capacity
constexpr int M_CAP = 4096;           // merge class capacity (one block per x)
constexpr int M2_CAP = 8192;          // larger merge class capacity
constexpr int M_THREADS = 256;       // threads per row of the merge classes above 2048 candidates
constexpr int M0_THREADS = 128;      // threads per row of the merge class up to 2048 candidates
constexpr int M_MAXL = 64;            // merge class: at most this many neighbour lists
constexpr int BM_THREADS = 1024;
constexpr int BM_MAX_WORDS = 52 * 1024;  // bitmap window: 208 KB + 6.5 KB summary + 12 KB counters/bounds
constexpr int BM_WARP_PER_LIST = 128;    // bitmap rows with this many neighbours are hubs (queued first)

enum { Q_WARP = 0, Q_W2 = 1, Q_COPY = 2, Q_BITMAP = 3, Q_MERGE = 4, Q_MERGE2 = 5, Q_HUB = 6,
       Q_MERGE0 = 7, NQ = 8 };
constexpr int64_t HUB_CAND = 65536;      // bitmap rows with this many candidates are hubs

struct Counters {
    unsigned long long cursor;        // scratch cursor
    unsigned long long need;          // scratch needed
    unsigned long long candidates;    // light join size
    uint32_t q[NQ];
    unsigned long long q_cand[NQ];    // candidates per class
    unsigned long long q_deg[NQ];     // neighbour-list entries read per class
    uint32_t bm_next;                 // bitmap kernel work counter (hubs, then the rest)
};

__device__ __forceinline__ uint32_t next_pow2(uint32_t v) {
    return v <= 1 ? 1u : 1u << (32 - __clz(v - 1));
}

// Per y, the neighbour list a light x and a heavy x read (light z only from a
// heavy y), so that the bitmap kernel finds a list's bounds with one load.
__global__ void ybounds_kernel(int64_t ny, const int32_t* __restrict__ syoff,
                               const int32_t* __restrict__ hy, const int32_t* __restrict__ sloff,
                               int2* __restrict__ ybl, int2* __restrict__ ybh) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < ny;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int2 l = make_int2(syoff[b], syoff[b + 1] - syoff[b]);
        ybl[b] = l;
        const int32_t j = hy[b];
        ybh[b] = j >= 0 ? make_int2(-sloff[j] - 1, sloff[j + 1] - sloff[j]) : l;
    }
}

// Candidate count c(x): a light x reads all of S[b] for its y, which the
// index build already summed (xsum; recomputed here when absent); a heavy x
// reads the lengths of the per-y lists it walks (ybh: light z only from a
// heavy y).  Lane per x; the x of a warp with more than 32 lists are summed by
// the whole warp, one after another.
__global__ void cand_kernel(int64_t nx, const int32_t* __restrict__ rxoff,
                            const int32_t* __restrict__ rycol, const int32_t* __restrict__ hx,
                            const int2* __restrict__ ybh, const int32_t* __restrict__ deg_sy,
                            const int64_t* __restrict__ xsum, int64_t* __restrict__ cand) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; base < nx;
         base += stride) {
        const int64_t a = base + lane;
        const bool valid = a < nx;
        int32_t e0 = 0, e1 = 0;
        bool heavy = false;
        if (valid) {
            e0 = rxoff[a];
            e1 = rxoff[a + 1];
            heavy = hx[a] >= 0;
        }
        const bool done = valid && !heavy && xsum;
        const bool small = valid && !done && e1 - e0 <= 32;
        long long c = done ? (long long)xsum[a] : 0;
        if (small) {
            int32_t e = e0;
            for (; e + 4 <= e1; e += 4) {        // four independent gathers in flight
                const int32_t b0 = rycol[e], b1 = rycol[e + 1], b2 = rycol[e + 2], b3 = rycol[e + 3];
                c += heavy ? (long long)ybh[b0].y + ybh[b1].y + ybh[b2].y + ybh[b3].y
                           : (long long)deg_sy[b0] + deg_sy[b1] + deg_sy[b2] + deg_sy[b3];
            }
            for (; e < e1; ++e) c += heavy ? ybh[rycol[e]].y : deg_sy[rycol[e]];
        }
        unsigned big = __ballot_sync(0xffffffffu, valid && !done && !small);
        while (big) {
            const int j = __ffs(big) - 1;
            big &= big - 1;
            const int32_t f0 = __shfl_sync(0xffffffffu, e0, j), f1 = __shfl_sync(0xffffffffu, e1, j);
            const bool hj = __shfl_sync(0xffffffffu, heavy, j);
            long long sj = 0;
            int32_t e = f0 + lane;
            for (; e + 7 * 32 < f1; e += 8 * 32) {   // eight independent chains per lane
                int32_t b[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) b[u] = rycol[e + 32 * u];
#pragma unroll
                for (int u = 0; u < 8; ++u) sj += hj ? ybh[b[u]].y : deg_sy[b[u]];
            }
            for (; e < f1; e += 32) sj += hj ? ybh[rycol[e]].y : deg_sy[rycol[e]];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sj += __shfl_xor_sync(0xffffffffu, sj, o);
            if (lane == j) c = sj;
        }
        if (valid) cand[a] = (int64_t)c;
    }
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Thread per x: class, queue slot (warp-aggregated atomics), block-aggregated sums.
// Scratch a row of x reserves: its distinct z can outnumber neither its
// light candidates c plus (heavy x) the w columns of its product row, nor all
// of its join candidates (xsum, summed over light and heavy y), nor |dom z|.
__device__ __forceinline__ unsigned long long row_bound(unsigned long long c, bool heavy,
                                                        int64_t w, int64_t nz,
                                                        const int64_t* xsum, int64_t a) {
    unsigned long long ub = c;
    if (heavy) {
        ub += (unsigned long long)w;
        if (xsum && ub > (unsigned long long)xsum[a]) ub = (unsigned long long)xsum[a];
    }
    return ub > (unsigned long long)nz ? (unsigned long long)nz : ub;
}

// A light x with a single neighbour list needs no deduplication: S[b] is
// sorted and distinct, so the output pass reads it in place (tmp_off holds
// -(offset in szval) - 1) and no scratch is used.
__global__ void queue_kernel(int64_t nx, const int64_t* cand, const int32_t* hx,
                             const int32_t* rxoff, const int32_t* rycol, const int32_t* syoff,
                             const int64_t* xsum, int64_t w, int64_t nz, int32_t* queues,
                             int32_t* cnt, int64_t* tmp_off, Counters* ctr) {
    __shared__ unsigned long long s_sum[2 + 2 * NQ];
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 2 + 2 * NQ; i += blockDim.x) s_sum[i] = 0;
    __syncthreads();
    unsigned long long need = 0, cands = 0, qc[NQ] = {}, qd[NQ] = {};
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nx;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = base + threadIdx.x;
        int q = -1;
        unsigned long long c = 0, ub = 0;
        if (a < nx) {
            const bool heavy = hx[a] >= 0;
            const int32_t dg = rxoff[a + 1] - rxoff[a];
            c = (unsigned long long)cand[a];
            if (!heavy && c > (unsigned long long)W_CAP && c <= (unsigned long long)M2_CAP &&
                dg > 1 && dg <= M_MAXL) {
                q = c <= (unsigned long long)W2_CAP ? Q_MERGE0
                                                    : (c <= (unsigned long long)M_CAP ? Q_MERGE : Q_MERGE2);
                ub = c;
            } else if (heavy || (c > (unsigned long long)W2_CAP && dg > 1)) {
                q = (dg >= BM_WARP_PER_LIST || c >= (unsigned long long)HUB_CAND) ? Q_HUB : Q_BITMAP;
                ub = row_bound(c, heavy, w, nz, xsum, a);
            } else if (c > 0 && rxoff[a + 1] - rxoff[a] == 1) {
                q = Q_COPY;
                cnt[a] = (int32_t)c;
                tmp_off[a] = -(int64_t)syoff[rycol[rxoff[a]]] - 1;
            } else if (c > 0) {
                q = c <= W_CAP ? Q_WARP : Q_W2;
                ub = c;
            }
            need += ub;
            cands += c;
            if (q >= 0) {
                qc[q] += c;
                qd[q] += (unsigned long long)(rxoff[a + 1] - rxoff[a]);
            }
        }
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const unsigned m = __ballot_sync(0xffffffffu, q == k);
            if (!m) continue;
            const int leader = __ffs(m) - 1;
            uint32_t pos = 0;
            if (lane == leader) pos = atomicAdd(&ctr->q[k], (uint32_t)__popc(m));
            pos = __shfl_sync(0xffffffffu, pos, leader);
            if (q == k) queues[(int64_t)k * nx + pos + __popc(m & ((1u << lane) - 1u))] = (int32_t)a;
        }
    }
    need = warp_sum(need);
    cands = warp_sum(cands);
    for (int k = 0; k < NQ; ++k) {
        qc[k] = warp_sum(qc[k]);
        qd[k] = warp_sum(qd[k]);
    }
    if (lane == 0) {
        atomicAdd(&s_sum[0], need);
        atomicAdd(&s_sum[1], cands);
        for (int k = 0; k < NQ; ++k) {
            atomicAdd(&s_sum[2 + k], qc[k]);
            atomicAdd(&s_sum[2 + NQ + k], qd[k]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_sum[0]) atomicAdd(&ctr->need, s_sum[0]);
        if (s_sum[1]) atomicAdd(&ctr->candidates, s_sum[1]);
        for (int k = 0; k < NQ; ++k) {
            if (s_sum[2 + k]) atomicAdd(&ctr->q_cand[k], s_sum[2 + k]);
            if (s_sum[2 + NQ + k]) atomicAdd(&ctr->q_deg[k], s_sum[2 + NQ + k]);
        }
    }
}

// ------------------------------------------------------------ bitonic sort
__device__ __forceinline__ void cswap(int32_t* k, uint32_t i, uint32_t p, bool up) {
    int32_t a = k[i], b = k[p];
    if ((a > b) == up) {
        k[i] = b;
        k[p] = a;
    }
}

__device__ void bitonic_warp(int32_t* k, uint32_t n) {
    const int lane = threadIdx.x & 31;
    for (uint32_t size = 2; size <= n; size <<= 1)
        for (uint32_t j = size >> 1; j > 0; j >>= 1) {
            for (uint32_t t = lane; t < n / 2; t += 32) {
                uint32_t i = 2 * t - (t & (j - 1));
                cswap(k, i, i + j, (i & size) == 0);
            }
            __syncwarp();
        }
}

template <typename T>
__device__ T block_exclusive(T v, T* sw, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sw[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T s = lane < nw ? sw[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sw[lane] = s;
    }
    __syncthreads();
    T prefix = warp > 0 ? sw[warp - 1] : T(0);
    *total = sw[nw - 1];
    __syncthreads();
    return prefix + x - v;
}

struct LightArgs {
    const int32_t* rxoff;
    const int32_t* rycol;
    const int32_t* syoff;
    const int32_t* szcol;
    const int32_t* szval;      // zval[szcol]: the lists of S as z values (same order)
    const int32_t* qbeg;       // batches: first x (= z) id of every query, else null
    int32_t nq;
    const int32_t* deg_sy;
    const int32_t* hx;
    const int32_t* hy;
    const int32_t* sloff;
    const int32_t* slcol;
    const int32_t* hz_inv;
    const uint32_t* G;
    int64_t g_stride;
    int64_t w;
    int64_t nz;
    const int64_t* cand;
    const int64_t* xsum;   // [nx] each x's join candidates over all its y (may be null)
    int32_t* tmp;
    int64_t tmp_cap;
    int64_t* tmp_off;
    int32_t* cnt;
    Counters* ctr;
    uint32_t* status;
    const int2* ybl;           // bitmap rows: per y, (start in szcol, length) of S[b]
    const int2* ybh;           // per y, the list a heavy x reads: light z of a heavy y as
                               // (-(offset in slcol) - 1, length), else as ybl
};

// ------------------------------------------------------------ warp classes
// One warp per light x: gather its candidates into a per-warp shared-memory
// buffer, bitonic-sort them, and write the distinct values in order.
template <int CAP>
__global__ void light_warp_kernel(LightArgs A, const int32_t* queue, const Counters* qc,
                                  int qid) {
    extern __shared__ int32_t dyn_keys[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int32_t* keys = dyn_keys + (size_t)wib * CAP;
    const uint32_t nq = qc->q[qid];
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t qi = warp; qi < nq; qi += nwarps) {
        const int32_t a = queue[qi];
        uint32_t off = 0;
        for (int32_t e = A.rxoff[a]; e < A.rxoff[a + 1]; ++e) {
            const int32_t b = A.rycol[e];
            const int32_t s0 = A.syoff[b], len = A.syoff[b + 1] - s0;
            for (int32_t t = lane; t < len; t += 32)
                if (off + t < CAP) keys[off + t] = A.szval[s0 + t];
            off += len;
        }
        if (off > CAP) {  // cannot happen: the class bound is the candidate count
            if (lane == 0) atomicOr(A.status, ST_BADINDEX);
            continue;
        }
        const uint32_t n = off;
        const uint32_t sz = max(32u, next_pow2(n));
        for (uint32_t t = n + lane; t < sz; t += 32) keys[t] = KEY_PAD;
        __syncwarp();
        bitonic_warp(keys, sz);
        uint32_t distinct = 0;
        for (uint32_t t = lane; t < ((n + 31) & ~31u); t += 32) {
            bool keep = t < n && (t == 0 || keys[t] != keys[t - 1]);
            distinct += __popc(__ballot_sync(0xffffffffu, keep));
        }
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&A.ctr->cursor, (unsigned long long)distinct);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base + distinct > (unsigned long long)A.tmp_cap) {
            if (lane == 0) atomicOr(A.status, ST_OVERFLOW);
            continue;
        }
        uint32_t pos = 0;
        for (uint32_t t = lane; t < ((n + 31) & ~31u); t += 32) {
            bool keep = t < n && (t == 0 || keys[t] != keys[t - 1]);
            unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) A.tmp[base + pos + __popc(m & ((1u << lane) - 1u))] = keys[t];
            pos += __popc(m);
        }
        if (lane == 0) {
            A.cnt[a] = (int32_t)distinct;
            A.tmp_off[a] = (int64_t)base;
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------ bucket class
// One warp per light x with W_CAP < c <= CAP, deduplicated by an
// order-preserving bucket sort: pass 1 counts the candidates per bucket of
// the row's z value range (bucket = (z - vlo) >> sh with span >> sh < nb,
// monotone; the range comes from the ends of the row's sorted lists),
// pass 2 scatters them to their bucket's range, then every lane sorts and
// deduplicates whole buckets (about 8 values each) by insertion, and the
// buckets are written in order.
// Work is linear in c; no block-wide synchronisation is needed.
template <int CAP, int NB>
__global__ void light_bucket_kernel(LightArgs A, const int32_t* queue, const Counters* qc,
                                    int qid) {
    extern __shared__ int32_t dyn_b[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int32_t* buf = dyn_b + (size_t)wib * (CAP + 2 * NB);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(buf + CAP);   // per-bucket count, later distinct
    uint32_t* cur = cnt + NB;                                 // per-bucket cursor / end
    const uint32_t nq = qc->q[qid];
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int PER = NB / 32;                              // counters per lane in scans
    for (int64_t qi = warp; qi < nq; qi += nwarps) {
        const int32_t a = queue[qi];
        const uint32_t n = (uint32_t)A.cand[a];
        if (n > CAP) {  // cannot happen: the class bound is the candidate count
            if (lane == 0) atomicOr(A.status, ST_BADINDEX);
            continue;
        }
        const uint32_t nb = min((uint32_t)NB, max(32u, next_pow2((n + 7) / 8)));
        for (uint32_t k = lane; k < NB; k += 32) cnt[k] = 0;
        const int32_t e0 = A.rxoff[a], e1 = A.rxoff[a + 1];
        // the row's value range from its sorted lists' first and last entries;
        // bucket = (z - vlo) >> sh is monotone in z and (span >> sh) < nb
        int32_t vlo = INT32_MAX, vhi = INT32_MIN;
        for (int32_t e = e0 + lane; e < e1; e += 32) {
            const int32_t b = A.rycol[e];
            const int32_t s0 = A.syoff[b], s1 = A.syoff[b + 1];
            if (s1 > s0) {
                vlo = min(vlo, A.szval[s0]);
                vhi = max(vhi, A.szval[s1 - 1]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vlo = min(vlo, __shfl_xor_sync(0xffffffffu, vlo, o));
            vhi = max(vhi, __shfl_xor_sync(0xffffffffu, vhi, o));
        }
        const uint32_t span = vhi >= vlo ? (uint32_t)vhi - (uint32_t)vlo : 0u;
        const int sh = max(0, (32 - __clz(span)) - (31 - __clz(nb)));
        __syncwarp();
        for (int32_t e = e0; e < e1; ++e) {
            const int32_t b = A.rycol[e];
            const int32_t s0 = A.syoff[b], L = A.syoff[b + 1] - s0;
            for (int32_t t0 = lane; t0 < L; t0 += 128) {
                int32_t zz[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) zz[u] = (t0 + 32 * u < L) ? A.szval[s0 + t0 + 32 * u] : 0;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (t0 + 32 * u < L) atomicAdd(&cnt[((uint32_t)zz[u] - (uint32_t)vlo) >> sh], 1u);
            }
        }
        __syncwarp();
        // exclusive scan of the counts into the cursors
        {
            uint32_t loc[PER], s = 0;
#pragma unroll
            for (int i = 0; i < PER; ++i) { loc[i] = cnt[lane * PER + i]; s += loc[i]; }
            uint32_t inc = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            uint32_t run = inc - s;
#pragma unroll
            for (int i = 0; i < PER; ++i) { cur[lane * PER + i] = run; run += loc[i]; }
        }
        __syncwarp();
        for (int32_t e = e0; e < e1; ++e) {
            const int32_t b = A.rycol[e];
            const int32_t s0 = A.syoff[b], L = A.syoff[b + 1] - s0;
            for (int32_t t0 = lane; t0 < L; t0 += 128) {
                int32_t zz[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) zz[u] = (t0 + 32 * u < L) ? A.szval[s0 + t0 + 32 * u] : 0;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (t0 + 32 * u < L) {
                        const uint32_t p = atomicAdd(&cur[((uint32_t)zz[u] - (uint32_t)vlo) >> sh], 1u);
                        buf[p] = zz[u];
                    }
            }
        }
        __syncwarp();
        // sort + deduplicate every bucket in place; cnt[k] becomes its distinct count
        for (uint32_t k = lane; k < nb; k += 32) {
            const uint32_t end = cur[k], beg = end - cnt[k];
            for (uint32_t i = beg + 1; i < end; ++i) {
                const int32_t v = buf[i];
                uint32_t j = i;
                while (j > beg && buf[j - 1] > v) { buf[j] = buf[j - 1]; --j; }
                buf[j] = v;
            }
            uint32_t d = 0;
            for (uint32_t i = beg; i < end; ++i)
                if (i == beg || buf[i] != buf[i - 1]) buf[beg + d++] = buf[i];
            cnt[k] = d;
        }
        __syncwarp();
        // positions of the buckets' distinct runs in the output
        uint32_t total;
        {
            uint32_t loc[PER], s = 0;
#pragma unroll
            for (int i = 0; i < PER; ++i) { loc[i] = (lane * PER + i < nb) ? cnt[lane * PER + i] : 0; s += loc[i]; }
            uint32_t inc = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            total = __shfl_sync(0xffffffffu, inc, 31);
            uint32_t run = inc - s;
            // cnt[k] becomes bucket k's output position (each lane rewrites
            // only the counters it read); cur[k] keeps the bucket's end in buf
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const uint32_t k = lane * PER + i;
                if (k < nb) {
                    cnt[k] = run;
                    run += loc[i];
                }
            }
        }
        __syncwarp();
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&A.ctr->cursor, (unsigned long long)total);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base + total > (unsigned long long)A.tmp_cap) {
            if (lane == 0) atomicOr(A.status, ST_OVERFLOW);
            continue;
        }
        // bucket k starts in buf where bucket k-1 ended; its distinct values
        // were compacted to that start, and their number is the gap between
        // consecutive output positions
        for (uint32_t k = lane; k < nb; k += 32) {
            const uint32_t outp = cnt[k];
            const uint32_t d = ((k + 1 < nb) ? cnt[k + 1] : total) - outp;
            const uint32_t beg = (k == 0) ? 0u : cur[k - 1];
            for (uint32_t i = 0; i < d; ++i) A.tmp[base + outp + i] = buf[beg + i];
        }
        if (lane == 0) {
            A.cnt[a] = (int32_t)total;
            A.tmp_off[a] = (int64_t)base;
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------ merge class
// One block per light x with W2_CAP < c <= M_CAP and 2..M_MAXL neighbour
// lists.  Every S[b] is already sorted, so the candidates are deg sorted runs:
// they are gathered into shared memory run after run, merged pairwise
// (ceil(log2 deg) levels; in each level every thread produces a fixed share of
// the outputs, starting at the co-rank found by a merge-path search), and the
// merged sequence is deduplicated by comparing neighbours.  Work is linear in
// c per level and the output is written with coalesced stores.
// number of elements of A among the first d outputs of merge(A, B), where
// ties take A first
__device__ __forceinline__ int32_t co_rank(const int32_t* A, int32_t la, const int32_t* B,
                                           int32_t lb, int32_t d) {
    int32_t lo = max(0, d - lb), hi = min(d, la);
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (A[mid] <= B[d - mid - 1]) lo = mid + 1; else hi = mid;
    }
    return lo;
}

template <int CAP, int TPB>
__global__ void __launch_bounds__(TPB)
    light_merge_kernel(LightArgs A, const int32_t* queue, const Counters* qc, int qid) {
    extern __shared__ int32_t dyn_m[];
    __shared__ int32_t s_runs[2][M_MAXL + 1];   // run boundaries, current and next level
    __shared__ int32_t s_start[M_MAXL];         // list starts in szval
    __shared__ uint32_t s_wsum[TPB / 32];
    __shared__ unsigned long long s_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nq = qc->q[qid];
    for (int64_t qi = blockIdx.x; qi < nq; qi += gridDim.x) {
        const int32_t a = queue[qi];
        const int32_t e0 = A.rxoff[a], deg = A.rxoff[a + 1] - e0;
        if (deg < 1 || deg > M_MAXL) {   // cannot happen: the class bounds the degree
            if (tid == 0) atomicOr(A.status, ST_BADINDEX);
            continue;
        }
        // run boundaries: warp 0, two lists per lane
        if (warp == 0) {
            int32_t L0 = 0, L1 = 0, st0 = 0, st1 = 0;
            const int i0 = 2 * lane, i1 = 2 * lane + 1;
            if (i0 < deg) {
                const int32_t b = A.rycol[e0 + i0];
                st0 = A.syoff[b];
                L0 = A.syoff[b + 1] - st0;
            }
            if (i1 < deg) {
                const int32_t b = A.rycol[e0 + i1];
                st1 = A.syoff[b];
                L1 = A.syoff[b + 1] - st1;
            }
            int32_t inc = L0 + L1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            const int32_t ex = inc - L0 - L1;
            if (lane == 0) s_runs[0][0] = 0;
            if (i0 < deg) { s_runs[0][i0 + 1] = ex + L0; s_start[i0] = st0; }
            if (i1 < deg) { s_runs[0][i1 + 1] = ex + L0 + L1; s_start[i1] = st1; }
        }
        __syncthreads();
        const int32_t c = s_runs[0][deg];
        if (c > CAP) {                   // cannot happen: the class bounds c
            if (tid == 0) atomicOr(A.status, ST_BADINDEX);
            __syncthreads();
            continue;
        }
        // the reservation (c slots, an upper bound of the distinct count) is
        // read only after the merge, so its latency overlaps it
        if (tid == 0) s_base = atomicAdd(&A.ctr->cursor, (unsigned long long)c);
        int32_t* src = dyn_m;
        int32_t* dst = dyn_m + CAP;
        // gather: flat candidate f of run k is S[b_k][f - run_k]; a thread's f
        // only grow, so its run index k only moves forward
        constexpr int U = 8;
        // the thread's current run: [r_beg, r_end) starting at S offset r_st,
        // kept in registers (shared memory is read only at run boundaries)
        int k = 0;
        int32_t r_beg = 0, r_end = s_runs[0][1], r_st = s_start[0];
        for (int32_t f0 = tid; f0 < c; f0 += U * TPB) {
            int32_t zz[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int32_t f = f0 + u * TPB;
                zz[u] = 0;
                if (f < c) {
                    while (r_end <= f) {
                        ++k;
                        r_beg = r_end;
                        r_end = s_runs[0][k + 1];
                        r_st = s_start[k];
                    }
                    zz[u] = A.szval[r_st + (f - r_beg)];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int32_t f = f0 + u * TPB;
                if (f < c) src[f] = zz[u];
            }
        }
        __syncthreads();
        // pairwise merge levels
        int runs = deg, cur = 0;
        // a thread's share of the outputs; odd, so that the 32 lanes' stores
        // (per words apart) fall in 32 different shared-memory banks
        const int32_t per = ((c + TPB - 1) / TPB) | 1;
        while (runs > 1) {
            const int32_t* rb = s_runs[cur];
            const int pairs = (runs + 1) >> 1;
            if (tid <= pairs) s_runs[cur ^ 1][tid] = tid < pairs ? rb[2 * tid] : c;
            int32_t o = min(c, tid * per);
            const int32_t o_end = min(c, o + per);
            while (o < o_end) {
                int lo = 0, hi = pairs;          // pair p with rb[2p] <= o < its end
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (rb[2 * mid] <= o) lo = mid; else hi = mid;
                }
                const int32_t a0 = rb[2 * lo], a1 = rb[min(2 * lo + 1, runs)],
                              b1 = rb[min(2 * lo + 2, runs)];
                const int32_t seg_end = min(o_end, b1);
                const int32_t i = co_rank(src + a0, a1 - a0, src + a1, b1 - a1, o - a0);
                int32_t ia = a0 + i, ib = a1 + (o - a0 - i);
                int32_t va = ia < a1 ? src[ia] : 0;
                int32_t vb = ib < b1 ? src[ib] : 0;
                for (; o < seg_end; ++o) {
                    // branch-free step: one shared-memory load per output; take A
                    // while it has values and (B is done or A's head is not larger)
                    const bool ta = ia < a1 && (ib >= b1 || va <= vb);
                    dst[o] = ta ? va : vb;
                    ia += ta;
                    ib += !ta;
                    const int32_t ni = ta ? ia : ib;
                    const int32_t nv = ni < (ta ? a1 : b1) ? src[ni] : 0;
                    va = ta ? nv : va;
                    vb = ta ? vb : nv;
                }
            }
            __syncthreads();
            int32_t* t = src;
            src = dst;
            dst = t;
            cur ^= 1;
            runs = pairs;
        }
        // deduplicate neighbours: warp w owns a range of whole 32-value rounds
        const int32_t rounds = (c + 31) >> 5;
        const int32_t rpw = (rounds + (TPB / 32) - 1) / (TPB / 32);
        const int32_t wb = min(c, warp * rpw * 32), we = min(c, wb + rpw * 32);
        uint32_t mine = 0;
        for (int32_t i = wb + lane; i - lane < we; i += 32) {
            const bool keep = i < we && (i == 0 || src[i] != src[i - 1]);
            mine += __popc(__ballot_sync(0xffffffffu, keep));
        }
        if (lane == 0) s_wsum[warp] = mine;
        __syncthreads();
        uint32_t before = 0, total = 0;
#pragma unroll
        for (int k = 0; k < TPB / 32; ++k) {
            const uint32_t v = s_wsum[k];
            before += k < warp ? v : 0u;
            total += v;
        }
        const unsigned long long base = s_base;
        const bool room = base + (unsigned long long)c <= (unsigned long long)A.tmp_cap;
        if (room) {
            uint32_t pos = before;
            for (int32_t i = wb + lane; i - lane < we; i += 32) {
                const bool keep = i < we && (i == 0 || src[i] != src[i - 1]);
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                if (keep) A.tmp[base + pos + __popc(m & ((1u << lane) - 1u))] = src[i];
                pos += __popc(m);
            }
        }
        if (tid == 0) {
            if (!room) atomicOr(A.status, ST_OVERFLOW);
            A.cnt[a] = room ? (int32_t)total : 0;
            A.tmp_off[a] = (int64_t)base;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ bitmap class
// Set bit r; a bit that was clear is a new distinct value of the row, counted
// for the thread that owns its word in the emission (owner_shift: log2 of the
// words a thread owns).
// Word wi of the bitmap is stored at wi ^ (its owner's thread index mod 32):
// in the emission walk all lanes of a warp visit the j-th word of their own
// 32-word groups at the same time, and this spreads them over the 32 banks
// (without it every lane reads bank j).  A warp reading a whole 32-word
// group reads a permutation of it, also conflict-free.
__device__ __forceinline__ int32_t bm_at(int32_t wi, int owner_shift) {
    return wi ^ ((wi >> owner_shift) & 31);
}

__device__ __forceinline__ void mark(uint32_t* bm, uint32_t* summ, uint32_t* own, int owner_shift,
                                     int32_t r) {
    const int32_t wi = r >> 5;
    const uint32_t bit = 1u << (r & 31);
    const uint32_t old = atomicOr(&bm[bm_at(wi, owner_shift)], bit);
    if (old == 0) atomicOr(&summ[wi >> 5], 1u << (wi & 31));
    if (!(old & bit)) atomicAdd(&own[wi >> owner_shift], 1u);
}

// Marking of one chunk of a row's lists.  Flat candidate f belongs to the
// last list k with s_pre[k] <= f (a STEPS-step binary search: the chunk has at
// most 2^STEPS lists, and entries past them hold the total).  Each warp takes
// one contiguous run of the chunk's candidates, lane i the candidates
// run_start + i, + 32, ..., so a lane's list only moves forward: the lane keeps
// its list's bounds in registers and reads shared memory only when a
// candidate is past them (one step forward when the next list holds it, else
// the search).  Each thread loads U candidates before it marks any.
template <int STEPS>
__device__ __forceinline__ int32_t chunk_list(const uint32_t* s_pre, uint32_t f) {
    int32_t k = 0;      // last k with s_pre[k] <= f (s_pre[0] = 0)
#pragma unroll
    for (int step = 1 << (STEPS - 1); step > 0; step >>= 1)
        if (s_pre[k + step] <= f) k += step;
    return k;
}
template <int STEPS>
__device__ __forceinline__ void mark_chunk(const LightArgs& A, const uint32_t* s_pre,
                                           const int32_t* s_start, uint32_t total, int64_t z0,
                                           int64_t zend, uint32_t* bm, uint32_t* summ,
                                           uint32_t* own, int owner_shift) {
    constexpr int U = 8, NW = BM_THREADS / 32, LAST = (1 << STEPS) - 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t per = ((total + NW - 1) / NW + 31) & ~31u;
    const uint32_t fb = min(total, (uint32_t)warp * per), fe = min(total, fb + per);
    if (fb + lane >= fe) return;
    // entries past the chunk's lists hold the total, so pn = total past the last list
    int32_t k = chunk_list<STEPS>(s_pre, fb + lane);
    uint32_t pk = s_pre[k], pn = k < LAST ? s_pre[k + 1] : total;
    int32_t sk = s_start[k];
    for (uint32_t g = fb + lane; g < fe; g += 32 * U) {
        int32_t zz[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t f = g + 32u * (uint32_t)u;
            zz[u] = -1;
            if (f < fe) {
                if (f >= pn) {
                    const uint32_t p2 = k + 1 < LAST ? s_pre[k + 2] : total;
                    k = f < p2 ? k + 1 : chunk_list<STEPS>(s_pre, f);
                    pk = s_pre[k];
                    pn = k < LAST ? s_pre[k + 1] : total;
                    sk = s_start[k];
                }
                const uint32_t off = f - pk;
                zz[u] = sk >= 0 ? A.szcol[sk + off] : A.slcol[-sk - 1 + off];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (zz[u] >= z0 && zz[u] < zend)
                mark(bm, summ, own, owner_shift, (int32_t)(zz[u] - z0));
    }
}

// Exclusive prefix over a 1024-thread block; *total gets the block's sum.
// Two barriers; sw holds 32 words.
__device__ __forceinline__ uint32_t bm_block_scan(uint32_t v, uint32_t* sw, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) sw[warp] = inc;
    __syncthreads();
    const uint32_t x = sw[lane];
    uint32_t before = lane < warp ? x : 0u, tot = x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        before += __shfl_xor_sync(0xffffffffu, before, o);
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    *total = tot;
    __syncthreads();
    return before + inc - v;
}

// Lane whose exclusive prefix ex starts the run holding j: the last lane with
// ex <= j (a lane whose count is 0 is never returned for j below the total).
__device__ __forceinline__ int run_owner(uint32_t ex, uint32_t j) {
    int owner = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const uint32_t e = __shfl_sync(0xffffffffu, ex, owner + step);
        if (e <= j) owner += step;
    }
    return owner;
}

// Persistent blocks of 1024 threads, one x at a time; the rows come from a
// work counter, hubs first.  Shared memory (dynamic): the bitmap window, its
// summary (one bit per non-zero bitmap word), a distinct-value counter per
// thread, and the current chunk's list bounds.  The bitmap, the summary and
// the counters start at zero and are cleared as they are emitted.
//
// Thread t owns the 32 * spt bitmap words of summary words [t * spt,
// (t + 1) * spt); its output run is their set bits in z order.  Marking
// counts every bit that goes from clear to set for the owning thread, so
// each thread knows its run's length without a pass over the bitmap.
//
// Marking: the row's neighbour lists are taken 1024 at a time, one per
// thread (bounds from the per-y tables, prefix-summed over the block); each
// warp then marks a contiguous run of the chunk's flat candidates (adjacent
// lanes read adjacent list entries), each lane holding its current list's
// bounds in registers (mark_chunk).  A heavy row's product row (bit l of G
// means (a, hz_inv[l]) is an output) is expanded by all warps, 32 words at a
// time.
// Emission: rows with up to BM_DENSE values are written by each thread
// walking its own words; denser rows by warps, each over the words of its 32
// threads, 32 words at a time with coalesced stores.
constexpr int BM_CHUNK = 1024;           // neighbour lists per marking chunk
static_assert(BM_CHUNK == 1 << 10, "the deepest marking search (10 steps) covers one chunk");
constexpr uint32_t BM_DENSE = 160000;    // rows with more values are emitted by warps

__global__ void __launch_bounds__(BM_THREADS, 1)
    light_bitmap_kernel(LightArgs A, const int32_t* hub_queue, const int32_t* queue,
                        const Counters* qc, int32_t win_words) {
    extern __shared__ uint32_t smem_bm[];
    uint32_t* bm = smem_bm;                          // win_words (a multiple of 32)
    uint32_t* summ = smem_bm + win_words;            // win_words / 32
    uint32_t* own = summ + win_words / 32;           // BM_THREADS
    uint32_t* s_pre = own + BM_THREADS;              // BM_CHUNK
    int32_t* s_start = reinterpret_cast<int32_t*>(s_pre + BM_CHUNK);   // BM_CHUNK
    __shared__ uint32_t sw[32];
    __shared__ unsigned long long s_base;
    __shared__ uint32_t s_item[2];             // work items of this row and the next
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nh = qc->q[Q_HUB], nq = nh + qc->q[Q_BITMAP];
    const int64_t win_bits = (int64_t)win_words * 32;
    const int32_t nsumm_win = win_words / 32;
    // words per thread: spt summary words, a power of two
    int32_t spt = 1, owner_shift = 5;
    while (spt * BM_THREADS < nsumm_win) {
        spt <<= 1;
        ++owner_shift;
    }
    for (int32_t i = threadIdx.x; i < win_words + nsumm_win + BM_THREADS; i += blockDim.x)
        smem_bm[i] = 0;
    if (threadIdx.x == 0) s_item[0] = atomicAdd(&A.ctr->bm_next, 1u);
    __syncthreads();
    for (uint32_t r = 0;; ++r) {
        const uint32_t qi = s_item[r & 1];
        if (qi >= nq) break;
        if (threadIdx.x == 0) s_item[(r + 1) & 1] = atomicAdd(&A.ctr->bm_next, 1u);
        const int32_t a = qi < nh ? hub_queue[qi] : queue[qi - nh];
        const int32_t h = A.hx[a];
        const bool heavy = h >= 0;
        const int2* yb = heavy ? A.ybh : A.ybl;
        const int32_t e0 = A.rxoff[a], deg = A.rxoff[a + 1] - e0;
        const unsigned long long ub =
            row_bound((unsigned long long)A.cand[a], heavy, A.w, A.nz, A.xsum, a);
        // read only after the marking phase's barriers: its latency overlaps them
        if (threadIdx.x == 0) s_base = atomicAdd(&A.ctr->cursor, ub);
        unsigned long long running = 0;
        bool room = true;
        unsigned long long base = 0;
        // the z ids a row can reach: its query's range in a batch (x and z ids
        // of one query coincide), else the whole domain
        int64_t zr0 = 0, zr1 = A.nz;
        if (A.qbeg) {
            int32_t lo = 0, hi = A.nq;          // last q with qbeg[q] <= a
            while (hi - lo > 1) {
                const int32_t mid = (lo + hi) >> 1;
                if (A.qbeg[mid] <= a) lo = mid; else hi = mid;
            }
            zr0 = A.qbeg[lo];
            zr1 = A.qbeg[lo + 1];
        }
        for (int64_t z0 = zr0; z0 < zr1; z0 += win_bits) {
            const int64_t zend = min(zr1, z0 + win_bits);
            const int32_t nwords = (int32_t)((zend - z0 + 31) >> 5);
            const int32_t nsumm = (nwords + 31) >> 5;
            // ---- mark the light candidates, 1024 neighbour lists at a time
            for (int32_t c0 = 0; c0 < deg; c0 += BM_CHUNK) {
                const int32_t n = min(BM_CHUNK, deg - c0);
                int2 bl = make_int2(0, 0);   // (start, length); start < 0: -(offset in slcol) - 1
                if ((int32_t)threadIdx.x < n) bl = yb[A.rycol[e0 + c0 + threadIdx.x]];
                uint32_t total;
                const uint32_t ex = bm_block_scan((uint32_t)bl.y, sw, &total);
                // entries past the chunk's lists hold the total, so the search
                // over all BM_CHUNK entries never selects them
                s_pre[threadIdx.x] = (int32_t)threadIdx.x < n ? ex : total;
                s_start[threadIdx.x] = bl.x;
                __syncthreads();
                // the search needs log2 of the chunk's list count rounded up
                // to a power of two: three unrolled depths
                if (n <= 32)
                    mark_chunk<5>(A, s_pre, s_start, total, z0, zend, bm, summ, own, owner_shift);
                else if (n <= 256)
                    mark_chunk<8>(A, s_pre, s_start, total, z0, zend, bm, summ, own, owner_shift);
                else
                    mark_chunk<10>(A, s_pre, s_start, total, z0, zend, bm, summ, own, owner_shift);
                __syncthreads();        // s_pre / s_start are rewritten by the next chunk
            }
            // ---- heavy product row, 32 words per warp step
            if (heavy && A.G) {
                const int32_t gw = (int32_t)((A.w + 31) >> 5);
                const uint32_t* grow = A.G + (int64_t)h * A.g_stride;
                for (int32_t i0 = warp * 32; i0 < gw; i0 += BM_THREADS) {
                    const int32_t i = i0 + lane;
                    const uint32_t wd = i < gw ? grow[i] : 0u;
                    const uint32_t c = __popc(wd);
                    uint32_t inc = c;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += y;
                    }
                    const uint32_t T = __shfl_sync(0xffffffffu, inc, 31), exl = inc - c;
                    for (uint32_t j0 = 0; j0 < T; j0 += 32) {
                        const uint32_t j = j0 + lane;
                        const int owner = run_owner(exl, j);
                        const uint32_t ow = __shfl_sync(0xffffffffu, wd, owner);
                        const uint32_t oe = __shfl_sync(0xffffffffu, exl, owner);
                        if (j < T) {
                            const int bt = (int)__fns(ow, 0u, (int)(j - oe) + 1);
                            const int64_t l = (int64_t)(i0 + owner) * 32 + bt;
                            if (l < A.w) {
                                const int64_t z = A.hz_inv[l];
                                if (z >= z0 && z < zend)
                                    mark(bm, summ, own, owner_shift, (int32_t)(z - z0));
                            }
                        }
                    }
                }
            }
            __syncthreads();
            // ---- emit the set bits in z order
            const uint32_t mine = own[threadIdx.x];
            own[threadIdx.x] = 0;
            uint32_t D;
            const uint32_t myex = bm_block_scan(mine, sw, &D);
            base = s_base;
            room = base + ub <= (unsigned long long)A.tmp_cap;
            if (!room && z0 == zr0 && threadIdx.x == 0) atomicOr(A.status, ST_OVERFLOW);
            const unsigned long long lim = base + ub;
            const int32_t slo = min(nsumm, (int32_t)threadIdx.x * spt);
            const int32_t shi = min(nsumm, slo + spt);
            if (D <= BM_DENSE) {
                unsigned long long p = base + running + myex;
                for (int32_t s = slo; s < shi; ++s) {
                    uint32_t m = summ[s];
                    summ[s] = 0;
                    while (m) {
                        const int j = __ffs(m) - 1;
                        m &= m - 1;
                        const int32_t wi = s * 32 + j;
                        const int32_t pw = bm_at(wi, owner_shift);
                        uint32_t bits = bm[pw];
                        bm[pw] = 0;
                        while (bits) {
                            const int bt = __ffs(bits) - 1;
                            bits &= bits - 1;
                            if (room && p < lim) A.tmp[p] = (int32_t)(z0 + (int64_t)wi * 32 + bt);
                            ++p;
                        }
                    }
                }
            } else {
                // the warp's words are those of its 32 threads; its run starts
                // where its first thread's does
                unsigned long long p = base + running + __shfl_sync(0xffffffffu, myex, 0);
                const int32_t g0 = min(nsumm, warp * 32 * spt);
                const int32_t g1 = min(nsumm, g0 + 32 * spt);
                for (int32_t g = g0; g < g1; ++g) {
                    if (summ[g] == 0) continue;
                    const int32_t wi = g * 32 + lane;
                    const int32_t pw = bm_at(wi, owner_shift);
                    const uint32_t wd = bm[pw];
                    bm[pw] = 0;
                    const uint32_t c = __popc(wd);
                    uint32_t inc = c;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += y;
                    }
                    const uint32_t T = __shfl_sync(0xffffffffu, inc, 31), exl = inc - c;
                    for (uint32_t j0 = 0; j0 < T; j0 += 32) {
                        const uint32_t j = j0 + lane;
                        const int owner = run_owner(exl, j);
                        const uint32_t ow = __shfl_sync(0xffffffffu, wd, owner);
                        const uint32_t oe = __shfl_sync(0xffffffffu, exl, owner);
                        if (j < T) {
                            const int bt = (int)__fns(ow, 0u, (int)(j - oe) + 1);
                            const unsigned long long o = p + j;
                            if (room && o < lim)
                                A.tmp[o] = (int32_t)(z0 + (int64_t)(g * 32 + owner) * 32 + bt);
                        }
                    }
                    p += T;
                    __syncwarp();
                    if (lane == 0) summ[g] = 0;
                }
            }
            running += D;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (running > ub) atomicOr(A.status, ST_BADINDEX);
            A.cnt[a] = room ? (int32_t)min(running, ub) : 0;
            A.tmp_off[a] = (int64_t)base | TMP_IDS;   // this list holds z ids
        }
    }
}

__global__ void szval_kernel(const int32_t* __restrict__ szcol, const int32_t* __restrict__ zval,
                             int64_t n, int32_t* __restrict__ szval) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        szval[i] = zval[szcol[i]];
}

}  // namespace

void light_and_union(const Graph& g, const Partition& p, const Heavy& h, LightResult& lr,
                     Arena& ws, cudaStream_t st, uint32_t* d_status, int64_t* host_scalars,
                     const int32_t* qbeg, int32_t nq) {
    (void)host_scalars;
    const int64_t nx = g.nx;
    lr.tmp_off = ws.get<int64_t>(nx + 1);
    lr.cnt = ws.get<int32_t>(nx + 1);
    JP_CUDA_TRY(cudaMemsetAsync(lr.cnt, 0, (nx + 1) * sizeof(int32_t), st));
    JP_CUDA_TRY(cudaMemsetAsync(lr.tmp_off, 0, (nx + 1) * sizeof(int64_t), st));
    if (nx == 0) return;
    int64_t* cand = ws.get<int64_t>(nx + 1);
    int32_t* queues = ws.get<int32_t>((size_t)NQ * nx);
    Counters* ctr = ws.get<Counters>(1);
    JP_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(Counters), st));
    tbegin(TM_CLASSIFY);
    // per y, the list a light x and a heavy x read (bounds for the bitmap
    // class, lengths for the candidate counts of heavy x)
    int2* ybl = ws.get<int2>((size_t)g.ny + 1);
    int2* ybh = ws.get<int2>((size_t)g.ny + 1);
    if (g.ny > 0) {
        ybounds_kernel<<<grid_for(g.ny, 256, 152 * 8), 256, 0, st>>>(g.ny, g.syoff, p.hy, p.sloff,
                                                                      ybl, ybh);
        JP_CHECK_LAUNCH();
    }
    cand_kernel<<<grid_for(nx, 256, 152 * 16), 256, 0, st>>>(
        nx, g.rxoff, g.rycol, p.hx, ybh, g.deg_sy, g.xsum, cand);
    JP_CHECK_LAUNCH();
    queue_kernel<<<grid_for(nx, 256, 152 * 8), 256, 0, st>>>(
        nx, cand, p.hx, g.rxoff, g.rycol, g.syoff, g.xsum, p.w, g.nz, queues, lr.cnt, lr.tmp_off,
        ctr);
    JP_CHECK_LAUNCH();
    tend(TM_CLASSIFY);
    Counters hc;
    JP_CUDA_TRY(cudaMemcpyAsync(&hc, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaStreamSynchronize(st));
    lr.candidates = (int64_t)hc.candidates;
    for (int q = 0; q < NQ; ++q) {
        lr.class_x[q] = hc.q[q];
        lr.class_cand[q] = (int64_t)hc.q_cand[q];
        lr.class_deg[q] = (int64_t)hc.q_deg[q];
    }
    lr.tmp_cap = (int64_t)hc.need;
    lr.tmp = ws.get<int32_t>((size_t)(lr.tmp_cap + 1));
    // the lists of S as z values: the sort and merge classes work on values
    // (ids are assigned in value order, so the order and the distinct sets
    // are the same) and write them, so output placement maps only bitmap rows
    lr.szval = ws.get<int32_t>((size_t)g.ns + 1);
    if (g.ns > 0) {
        szval_kernel<<<grid_for(g.ns, 256, 152 * 8), 256, 0, st>>>(g.szcol, g.zval, g.ns, lr.szval);
        JP_CHECK_LAUNCH();
    }

    LightArgs A;
    A.rxoff = g.rxoff;
    A.rycol = g.rycol;
    A.syoff = g.syoff;
    A.szcol = g.szcol;
    A.szval = lr.szval;
    A.qbeg = qbeg;
    A.nq = nq;
    A.deg_sy = g.deg_sy;
    A.hx = p.hx;
    A.hy = p.hy;
    A.sloff = p.sloff;
    A.slcol = p.slcol;
    A.hz_inv = p.hz_inv;
    A.G = h.present ? h.G : nullptr;
    A.g_stride = h.g_stride;
    A.w = p.w;
    A.nz = g.nz;
    A.cand = cand;
    A.xsum = g.xsum;
    A.tmp = lr.tmp;
    A.tmp_cap = lr.tmp_cap;
    A.tmp_off = lr.tmp_off;
    A.cnt = lr.cnt;
    A.ctr = ctr;
    A.status = d_status;
    A.ybl = nullptr;
    A.ybh = nullptr;

    if (hc.q[Q_WARP]) {
        const size_t sm = (size_t)8 * W_CAP * sizeof(int32_t);
        tbegin(TM_LIGHT_WARP);
        light_warp_kernel<W_CAP><<<grid_for((int64_t)hc.q[Q_WARP] * 32, 256, 152 * 16), 256, sm, st>>>(
            A, queues + (int64_t)Q_WARP * nx, ctr, Q_WARP);
        JP_CHECK_LAUNCH();
        tend(TM_LIGHT_WARP);
    }
    if (hc.q[Q_W2]) {
        constexpr int NB = 256;
        // 4 warps per block, (CAP + 2 NB) ints each: 40 KB, 5 blocks per SM
        const size_t sm = (size_t)4 * (W2_CAP + 2 * NB) * sizeof(int32_t);
        tbegin(TM_LIGHT_C2);
        light_bucket_kernel<W2_CAP, NB><<<grid_for((int64_t)hc.q[Q_W2] * 32, 128, 152 * 5), 128, sm, st>>>(
            A, queues + (int64_t)Q_W2 * nx, ctr, Q_W2);
        JP_CHECK_LAUNCH();
        tend(TM_LIGHT_C2);
    }
    if (hc.q[Q_MERGE0] || hc.q[Q_MERGE] || hc.q[Q_MERGE2]) {
        // 2 CAP ints of shared memory per block: 32 KB (6 blocks per SM) and
        // 64 KB (3 blocks per SM)
        const size_t sm0 = (size_t)2 * W2_CAP * sizeof(int32_t);   // 16 KB: 8 blocks per SM
        const size_t sm1 = (size_t)2 * M_CAP * sizeof(int32_t);
        const size_t sm2 = (size_t)2 * M2_CAP * sizeof(int32_t);
        smem_limit((const void*)light_merge_kernel<M_CAP, M_THREADS>, sm1);
        smem_limit((const void*)light_merge_kernel<M2_CAP, M_THREADS>, sm2);
        tbegin(TM_LIGHT_MERGE);
        if (hc.q[Q_MERGE2]) {
            light_merge_kernel<M2_CAP, M_THREADS><<<grid_for(hc.q[Q_MERGE2], 1, 152 * 3), M_THREADS, sm2, st>>>(
                A, queues + (int64_t)Q_MERGE2 * nx, ctr, Q_MERGE2);
            JP_CHECK_LAUNCH();
        }
        if (hc.q[Q_MERGE]) {
            light_merge_kernel<M_CAP, M_THREADS><<<grid_for(hc.q[Q_MERGE], 1, 152 * 6), M_THREADS, sm1, st>>>(
                A, queues + (int64_t)Q_MERGE * nx, ctr, Q_MERGE);
            JP_CHECK_LAUNCH();
        }
        if (hc.q[Q_MERGE0]) {
            light_merge_kernel<W2_CAP, M0_THREADS><<<grid_for(hc.q[Q_MERGE0], 1, 152 * 12), M0_THREADS, sm0, st>>>(
                A, queues + (int64_t)Q_MERGE0 * nx, ctr, Q_MERGE0);
            JP_CHECK_LAUNCH();
        }
        tend(TM_LIGHT_MERGE);
    }
    if (hc.q[Q_BITMAP] + hc.q[Q_HUB]) {
        A.ybl = ybl;
        A.ybh = ybh;
        int64_t words = (g.nz + 31) / 32;
        int32_t win = (int32_t)std::min<int64_t>(words, BM_MAX_WORDS);
        win = (win + 31) & ~31;                     // whole summary words
        const size_t sm = (size_t)(win + win / 32 + BM_THREADS + 2 * BM_CHUNK) * sizeof(uint32_t);
        smem_limit((const void*)light_bitmap_kernel,
                   (BM_MAX_WORDS + BM_MAX_WORDS / 32 + BM_THREADS + 2 * BM_CHUNK) * sizeof(uint32_t));
        tbegin(TM_LIGHT_BITMAP);
        light_bitmap_kernel<<<grid_for(hc.q[Q_BITMAP] + hc.q[Q_HUB], 1, 152), BM_THREADS, sm, st>>>(
            A, queues + (int64_t)Q_HUB * nx, queues + (int64_t)Q_BITMAP * nx, ctr, win);
        JP_CHECK_LAUNCH();
        tend(TM_LIGHT_BITMAP);
    }
}

}  // namespace jp
