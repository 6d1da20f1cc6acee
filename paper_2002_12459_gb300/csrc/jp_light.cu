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
//   c <= 256      a warp sorts the candidates in shared memory (bitonic)
//   c <= 2048     a 256-thread block sorts them
//   c <= 16384    a 1024-thread block sorts them
//   larger, and every heavy x: a block marks z in a shared-memory bitmap
//                 over the z domain (windowed when the domain is larger than
//                 shared memory); heavy rows also OR in their row of the
//                 heavy product bitmap G, which performs the union with the
//                 matrix part.  The set bits are emitted in z order.
// Each x's sorted distinct list goes to a scratch buffer at an offset taken
// by one atomic add; the output pass then places the lists in x order.
#include "jp_internal.cuh"

namespace jp {
namespace {

constexpr int32_t KEY_PAD = 0x7fffffff;
constexpr int W_CAP = 256;          // warp class capacity
constexpr int C2_CAP = 2048;        // 256-thread class capacity
constexpr int C16_CAP = 16384;      // 1024-thread class capacity
constexpr int BM_THREADS = 1024;
constexpr int BM_MAX_WORDS = 56 * 1024;   // 224 KB bitmap window (1,835,008 z values)

enum { Q_WARP = 0, Q_C2 = 1, Q_C16 = 2, Q_BITMAP = 3, NQ = 4 };

struct Counters {
    unsigned long long cursor;        // scratch cursor
    unsigned long long need;          // scratch needed
    unsigned long long candidates;    // light join size
    uint32_t q[NQ];
    unsigned long long q_cand[NQ];    // candidates per class
    unsigned long long q_deg[NQ];     // neighbour-list entries read per class
};

__device__ __forceinline__ uint32_t next_pow2(uint32_t v) {
    return v <= 1 ? 1u : 1u << (32 - __clz(v - 1));
}

__device__ __forceinline__ int64_t cand_of(int32_t b, bool heavy, const int32_t* hy,
                                           const int32_t* sloff, const int32_t* deg_sy) {
    if (heavy) {
        int32_t j = hy[b];
        if (j >= 0) return sloff[j + 1] - sloff[j];
    }
    return deg_sy[b];
}

// Warp per x: candidate count, class, scratch requirement.
__global__ void classify_kernel(int64_t nx, const int32_t* rxoff, const int32_t* rycol,
                                const int32_t* hx, const int32_t* hy, const int32_t* sloff,
                                const int32_t* deg_sy, int64_t w, int64_t nz, int64_t* cand,
                                int32_t* queues, Counters* ctr) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = warp; a < nx; a += nwarps) {
        const bool heavy = hx[a] >= 0;
        unsigned long long c = 0;
        for (int32_t e = rxoff[a] + lane; e < rxoff[a + 1]; e += 32)
            c += (unsigned long long)cand_of(rycol[e], heavy, hy, sloff, deg_sy);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if (lane == 0) {
            cand[a] = (int64_t)c;
            int q;
            unsigned long long ub;
            if (heavy || c > (unsigned long long)C16_CAP) {
                q = Q_BITMAP;
                ub = c + (heavy ? (unsigned long long)w : 0ull);
                if (ub > (unsigned long long)nz) ub = (unsigned long long)nz;
            } else if (c == 0) {
                q = -1;
                ub = 0;
            } else {
                q = c <= W_CAP ? Q_WARP : (c <= C2_CAP ? Q_C2 : Q_C16);
                ub = c;
            }
            if (q >= 0) {
                uint32_t pos = atomicAdd(&ctr->q[q], 1u);
                queues[(int64_t)q * nx + pos] = (int32_t)a;
                atomicAdd(&ctr->q_cand[q], c);
                atomicAdd(&ctr->q_deg[q], (unsigned long long)(rxoff[a + 1] - rxoff[a]));
            }
            if (ub) atomicAdd(&ctr->need, ub);
            if (c) atomicAdd(&ctr->candidates, c);
        }
    }
}

// ------------------------------------------------------------ bitonic sorts
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

__device__ void bitonic_block(int32_t* k, uint32_t n) {
    for (uint32_t size = 2; size <= n; size <<= 1)
        for (uint32_t j = size >> 1; j > 0; j >>= 1) {
            for (uint32_t t = threadIdx.x; t < n / 2; t += blockDim.x) {
                uint32_t i = 2 * t - (t & (j - 1));
                cswap(k, i, i + j, (i & size) == 0);
            }
            __syncthreads();
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
    int32_t* tmp;
    int64_t tmp_cap;
    int64_t* tmp_off;
    int32_t* cnt;
    Counters* ctr;
    uint32_t* status;
};

// ------------------------------------------------------------ warp class
__global__ void light_warp_kernel(LightArgs A, const int32_t* queue, const Counters* qc) {
    __shared__ int32_t keys_all[8][W_CAP];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int32_t* keys = keys_all[wib];
    const uint32_t nq = qc->q[Q_WARP];
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t qi = warp; qi < nq; qi += nwarps) {
        const int32_t a = queue[qi];
        uint32_t off = 0;
        for (int32_t e = A.rxoff[a]; e < A.rxoff[a + 1]; ++e) {
            const int32_t b = A.rycol[e];
            const int32_t s0 = A.syoff[b], len = A.syoff[b + 1] - s0;
            for (int32_t t = lane; t < len; t += 32)
                if (off + t < W_CAP) keys[off + t] = A.szcol[s0 + t];
            off += len;
        }
        if (off > W_CAP) {  // cannot happen: the class bound is the candidate count
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

// ------------------------------------------------------------ block classes
// Gather the candidates of a light x into keys[0..n); returns n.
__device__ uint32_t gather_block(const LightArgs& A, int32_t a, int32_t* keys, uint32_t cap,
                                 int32_t* nb_b, int32_t* nb_off, uint32_t* sw) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int32_t e0 = A.rxoff[a], deg = A.rxoff[a + 1] - e0;
    uint32_t base = 0;
    for (int32_t chunk = 0; chunk < deg; chunk += blockDim.x) {
        const int32_t i = chunk + threadIdx.x;
        int32_t b = -1;
        uint32_t len = 0;
        if (i < deg) {
            b = A.rycol[e0 + i];
            len = (uint32_t)A.deg_sy[b];
        }
        uint32_t tot;
        uint32_t ex = block_exclusive<uint32_t>(len, sw, &tot);
        nb_b[threadIdx.x] = b;
        nb_off[threadIdx.x] = (int32_t)(base + ex);
        __syncthreads();
        const int32_t cnt = min((int32_t)blockDim.x, deg - chunk);
        for (int32_t t = warp; t < cnt; t += nw) {
            const int32_t bb = nb_b[t];
            const int32_t s0 = A.syoff[bb], L = A.syoff[bb + 1] - s0;
            const uint32_t dst = (uint32_t)nb_off[t];
            for (int32_t q = lane; q < L; q += 32)
                if (dst + q < cap) keys[dst + q] = A.szcol[s0 + q];
        }
        base += tot;
        __syncthreads();
    }
    return base;
}

template <int CAP>
__global__ void light_block_kernel(LightArgs A, const int32_t* queue, const Counters* qc, int qid) {
    extern __shared__ int32_t dyn[];
    int32_t* keys = dyn;                       // CAP
    int32_t* nb_b = dyn + CAP;                 // blockDim
    int32_t* nb_off = nb_b + blockDim.x;       // blockDim
    __shared__ uint32_t sw[32];
    __shared__ unsigned long long s_base;
    const uint32_t nq = qc->q[qid];
    for (int64_t qi = blockIdx.x; qi < nq; qi += gridDim.x) {
        const int32_t a = queue[qi];
        const uint32_t n = gather_block(A, a, keys, CAP, nb_b, nb_off, sw);
        if (n > CAP) {
            if (threadIdx.x == 0) atomicOr(A.status, ST_BADINDEX);
            __syncthreads();
            continue;
        }
        const uint32_t sz = max(64u, next_pow2(n));
        for (uint32_t t = n + threadIdx.x; t < sz; t += blockDim.x) keys[t] = KEY_PAD;
        __syncthreads();
        bitonic_block(keys, sz);
        // distinct values: blocked ranges per thread
        const uint32_t ipt = (n + blockDim.x - 1) / blockDim.x;
        const uint32_t lo = min(n, threadIdx.x * ipt), hi = min(n, lo + ipt);
        uint32_t mine = 0;
        for (uint32_t t = lo; t < hi; ++t) mine += (t == 0 || keys[t] != keys[t - 1]);
        uint32_t tot;
        uint32_t ex = block_exclusive<uint32_t>(mine, sw, &tot);
        if (threadIdx.x == 0) s_base = atomicAdd(&A.ctr->cursor, (unsigned long long)tot);
        __syncthreads();
        const unsigned long long base = s_base;
        if (base + tot > (unsigned long long)A.tmp_cap) {
            if (threadIdx.x == 0) atomicOr(A.status, ST_OVERFLOW);
        } else {
            uint32_t p = ex;
            for (uint32_t t = lo; t < hi; ++t)
                if (t == 0 || keys[t] != keys[t - 1]) A.tmp[base + p++] = keys[t];
            if (threadIdx.x == 0) {
                A.cnt[a] = (int32_t)tot;
                A.tmp_off[a] = (int64_t)base;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ bitmap class
__global__ void __launch_bounds__(BM_THREADS, 1)
    light_bitmap_kernel(LightArgs A, const int32_t* queue, const Counters* qc, int32_t win_words) {
    extern __shared__ uint32_t bm[];
    __shared__ uint32_t sw[32];
    __shared__ unsigned long long s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t nq = qc->q[Q_BITMAP];
    const int64_t win_bits = (int64_t)win_words * 32;
    for (int64_t qi = blockIdx.x; qi < nq; qi += gridDim.x) {
        const int32_t a = queue[qi];
        const int32_t h = A.hx[a];
        const bool heavy = h >= 0;
        const int32_t e0 = A.rxoff[a], deg = A.rxoff[a + 1] - e0;
        unsigned long long ub = (unsigned long long)A.cand[a] +
                                (heavy ? (unsigned long long)A.w : 0ull);
        if (ub > (unsigned long long)A.nz) ub = (unsigned long long)A.nz;
        if (threadIdx.x == 0) s_base = atomicAdd(&A.ctr->cursor, ub);
        __syncthreads();
        const unsigned long long base = s_base;
        const bool room = base + ub <= (unsigned long long)A.tmp_cap;
        if (!room && threadIdx.x == 0) atomicOr(A.status, ST_OVERFLOW);
        unsigned long long running = 0;
        for (int64_t z0 = 0; z0 < A.nz; z0 += win_bits) {
            const int64_t zend = min(A.nz, z0 + win_bits);
            const int32_t nwords = (int32_t)((zend - z0 + 31) >> 5);
            for (int32_t i = threadIdx.x; i < nwords; i += blockDim.x) bm[i] = 0;
            __syncthreads();
            // light candidates, one warp per neighbour b
            for (int32_t t = warp; t < deg; t += nw) {
                const int32_t b = A.rycol[e0 + t];
                const int32_t* list;
                int32_t L;
                const int32_t j = heavy ? A.hy[b] : -1;
                if (j >= 0) {
                    list = A.slcol + A.sloff[j];
                    L = A.sloff[j + 1] - A.sloff[j];
                } else {
                    list = A.szcol + A.syoff[b];
                    L = A.syoff[b + 1] - A.syoff[b];
                }
                for (int32_t q = lane; q < L; q += 32) {
                    const int64_t z = list[q];
                    if (z >= z0 && z < zend) {
                        const int32_t r = (int32_t)(z - z0);
                        atomicOr(&bm[r >> 5], 1u << (r & 31));
                    }
                }
            }
            // heavy product row: bit l of G[h] means (a, hz_inv[l]) is an output
            if (heavy && A.G) {
                const int32_t gw = (int32_t)((A.w + 31) >> 5);
                const uint32_t* grow = A.G + (int64_t)h * A.g_stride;
                for (int32_t i = threadIdx.x; i < gw; i += blockDim.x) {
                    uint32_t bits = grow[i];
                    while (bits) {
                        const int bt = __ffs(bits) - 1;
                        bits &= bits - 1;
                        const int64_t l = (int64_t)i * 32 + bt;
                        if (l < A.w) {
                            const int64_t z = A.hz_inv[l];
                            if (z >= z0 && z < zend) {
                                const int32_t r = (int32_t)(z - z0);
                                atomicOr(&bm[r >> 5], 1u << (r & 31));
                            }
                        }
                    }
                }
            }
            __syncthreads();
            // emit set bits in z order
            const int32_t wpt = (nwords + blockDim.x - 1) / blockDim.x;
            const int32_t lo = min(nwords, (int32_t)threadIdx.x * wpt);
            const int32_t hi = min(nwords, lo + wpt);
            uint32_t mine = 0;
            for (int32_t i = lo; i < hi; ++i) mine += __popc(bm[i]);
            uint32_t tot;
            const uint32_t ex = block_exclusive<uint32_t>(mine, sw, &tot);
            if (room) {
                unsigned long long p = base + running + ex;
                const unsigned long long lim = base + ub;
                for (int32_t i = lo; i < hi; ++i) {
                    uint32_t bits = bm[i];
                    while (bits) {
                        const int bt = __ffs(bits) - 1;
                        bits &= bits - 1;
                        if (p < lim) A.tmp[p] = (int32_t)(z0 + (int64_t)i * 32 + bt);
                        ++p;
                    }
                }
            }
            running += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (running > ub) atomicOr(A.status, ST_BADINDEX);
            A.cnt[a] = room ? (int32_t)min(running, ub) : 0;
            A.tmp_off[a] = (int64_t)base;
        }
        __syncthreads();
    }
}

}  // namespace

void light_and_union(const Graph& g, const Partition& p, const Heavy& h, LightResult& lr,
                     Arena& ws, cudaStream_t st, uint32_t* d_status, int64_t* host_scalars) {
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
    classify_kernel<<<grid_for(nx * 32, 256, 152 * 16), 256, 0, st>>>(
        nx, g.rxoff, g.rycol, p.hx, p.hy, p.sloff, g.deg_sy, p.w, g.nz, cand, queues, ctr);
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

    LightArgs A;
    A.rxoff = g.rxoff;
    A.rycol = g.rycol;
    A.syoff = g.syoff;
    A.szcol = g.szcol;
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
    A.tmp = lr.tmp;
    A.tmp_cap = lr.tmp_cap;
    A.tmp_off = lr.tmp_off;
    A.cnt = lr.cnt;
    A.ctr = ctr;
    A.status = d_status;

    if (hc.q[Q_WARP]) {
        tbegin(TM_LIGHT_WARP);
        light_warp_kernel<<<grid_for((int64_t)hc.q[Q_WARP] * 32, 256, 152 * 16), 256, 0, st>>>(
            A, queues + (int64_t)Q_WARP * nx, ctr);
        JP_CHECK_LAUNCH();
        tend(TM_LIGHT_WARP);
    }
    if (hc.q[Q_C2]) {
        const size_t sm = (C2_CAP + 2 * 256) * sizeof(int32_t);
        tbegin(TM_LIGHT_C2);
        light_block_kernel<C2_CAP><<<grid_for(hc.q[Q_C2], 1, 152 * 8), 256, sm, st>>>(
            A, queues + (int64_t)Q_C2 * nx, ctr, Q_C2);
        JP_CHECK_LAUNCH();
        tend(TM_LIGHT_C2);
    }
    if (hc.q[Q_C16]) {
        const size_t sm = (C16_CAP + 2 * 1024) * sizeof(int32_t);
        static bool attr16 = false;
        if (!attr16) {
            JP_CUDA_TRY(cudaFuncSetAttribute(light_block_kernel<C16_CAP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            attr16 = true;
        }
        tbegin(TM_LIGHT_C16);
        light_block_kernel<C16_CAP><<<grid_for(hc.q[Q_C16], 1, 152 * 2), 1024, sm, st>>>(
            A, queues + (int64_t)Q_C16 * nx, ctr, Q_C16);
        JP_CHECK_LAUNCH();
        tend(TM_LIGHT_C16);
    }
    if (hc.q[Q_BITMAP]) {
        int64_t words = (g.nz + 31) / 32;
        int32_t win = (int32_t)std::min<int64_t>(words, BM_MAX_WORDS);
        win = (win + 31) & ~31;
        const size_t sm = (size_t)win * sizeof(uint32_t);
        static bool attrb = false;
        if (!attrb) {
            JP_CUDA_TRY(cudaFuncSetAttribute(light_bitmap_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(BM_MAX_WORDS * sizeof(uint32_t))));
            attrb = true;
        }
        tbegin(TM_LIGHT_BITMAP);
        light_bitmap_kernel<<<grid_for(hc.q[Q_BITMAP], 1, 152), BM_THREADS, sm, st>>>(
            A, queues + (int64_t)Q_BITMAP * nx, ctr, win);
        JP_CHECK_LAUNCH();
        tend(TM_LIGHT_BITMAP);
    }
}

}  // namespace jp
