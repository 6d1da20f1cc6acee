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
//   c <= 2048     a warp sorts them in a larger shared-memory buffer
//   larger, and every heavy x: a block marks z in a shared-memory bitmap
//                 over the z domain (windowed when the domain is larger than
//                 shared memory) with a one-bit-per-word summary, so that
//                 emitting and clearing cost grows with the touched words,
//                 not with the domain.  Heavy rows also OR in their row of
//                 the heavy product bitmap G: this is the union with the
//                 matrix part.  Set bits are emitted in z order.
// Each x's sorted distinct list goes to a scratch buffer at an offset taken
// by one atomic add; the output pass then places the lists in x order.
#include "jp_internal.cuh"

namespace jp {
namespace {

constexpr int32_t KEY_PAD = 0x7fffffff;
constexpr int W_CAP = 256;            // small warp class capacity
constexpr int W2_CAP = 2048;          // large warp class capacity
constexpr int BM_THREADS = 1024;
constexpr int BM_MAX_WORDS = 54 * 1024;  // bitmap window: 216 KB + 6.75 KB summary

enum { Q_WARP = 0, Q_W2 = 1, Q_UNUSED = 2, Q_BITMAP = 3, NQ = 4 };

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

// Warp per x: candidate count c(x).
__global__ void cand_kernel(int64_t nx, const int32_t* rxoff, const int32_t* rycol,
                            const int32_t* hx, const int32_t* hy, const int32_t* sloff,
                            const int32_t* deg_sy, int64_t* cand) {
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
        if (lane == 0) cand[a] = (int64_t)c;
    }
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Thread per x: class, queue slot (warp-aggregated atomics), block-aggregated sums.
__global__ void queue_kernel(int64_t nx, const int64_t* cand, const int32_t* hx,
                             const int32_t* rxoff, int64_t w, int64_t nz, int32_t* queues,
                             Counters* ctr) {
    __shared__ unsigned long long s_sum[2 + 2 * NQ];
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 2 + 2 * NQ; i += blockDim.x) s_sum[i] = 0;
    __syncthreads();
    unsigned long long need = 0, cands = 0, qc[NQ] = {0, 0, 0, 0}, qd[NQ] = {0, 0, 0, 0};
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nx;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = base + threadIdx.x;
        int q = -1;
        unsigned long long c = 0, ub = 0;
        if (a < nx) {
            const bool heavy = hx[a] >= 0;
            c = (unsigned long long)cand[a];
            if (heavy || c > (unsigned long long)W2_CAP) {
                q = Q_BITMAP;
                ub = c + (heavy ? (unsigned long long)w : 0ull);
                if (ub > (unsigned long long)nz) ub = (unsigned long long)nz;
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
                if (off + t < CAP) keys[off + t] = A.szcol[s0 + t];
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

// ------------------------------------------------------------ bitmap class
__device__ __forceinline__ void mark(uint32_t* bm, uint32_t* summ, int32_t r) {
    const int32_t wi = r >> 5;
    const uint32_t old = atomicOr(&bm[wi], 1u << (r & 31));
    if (old == 0) atomicOr(&summ[wi >> 5], 1u << (wi & 31));
}

// Persistent blocks, one x at a time.  The bitmap and its summary start at
// zero and are cleared word by word as they are emitted.
__global__ void __launch_bounds__(BM_THREADS, 1)
    light_bitmap_kernel(LightArgs A, const int32_t* queue, const Counters* qc, int32_t win_words) {
    extern __shared__ uint32_t smem_bm[];
    uint32_t* bm = smem_bm;                       // win_words
    uint32_t* summ = smem_bm + win_words;         // win_words / 32
    __shared__ uint32_t sw[32];
    __shared__ unsigned long long s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t nq = qc->q[Q_BITMAP];
    const int64_t win_bits = (int64_t)win_words * 32;
    for (int32_t i = threadIdx.x; i < win_words + win_words / 32; i += blockDim.x) smem_bm[i] = 0;
    __syncthreads();
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
            const int32_t nsumm = (nwords + 31) >> 5;
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
                    if (z >= z0 && z < zend) mark(bm, summ, (int32_t)(z - z0));
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
                            if (z >= z0 && z < zend) mark(bm, summ, (int32_t)(z - z0));
                        }
                    }
                }
            }
            __syncthreads();
            // emit set bits in z order: blocked ranges of summary words
            const int32_t spt = (nsumm + blockDim.x - 1) / blockDim.x;
            const int32_t lo = min(nsumm, (int32_t)threadIdx.x * spt);
            const int32_t hi = min(nsumm, lo + spt);
            uint32_t mine = 0;
            for (int32_t s = lo; s < hi; ++s) {
                uint32_t sm = summ[s];
                while (sm) {
                    const int j = __ffs(sm) - 1;
                    sm &= sm - 1;
                    mine += __popc(bm[s * 32 + j]);
                }
            }
            uint32_t tot;
            const uint32_t ex = block_exclusive<uint32_t>(mine, sw, &tot);
            unsigned long long p = base + running + ex;
            const unsigned long long lim = base + ub;
            for (int32_t s = lo; s < hi; ++s) {
                uint32_t sm = summ[s];
                summ[s] = 0;
                while (sm) {
                    const int j = __ffs(sm) - 1;
                    sm &= sm - 1;
                    const int32_t wi = s * 32 + j;
                    uint32_t bits = bm[wi];
                    bm[wi] = 0;
                    while (bits) {
                        const int bt = __ffs(bits) - 1;
                        bits &= bits - 1;
                        if (room && p < lim) A.tmp[p] = (int32_t)(z0 + (int64_t)wi * 32 + bt);
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
    cand_kernel<<<grid_for(nx * 32, 256, 152 * 16), 256, 0, st>>>(
        nx, g.rxoff, g.rycol, p.hx, p.hy, p.sloff, g.deg_sy, cand);
    JP_CHECK_LAUNCH();
    queue_kernel<<<grid_for(nx, 256, 152 * 8), 256, 0, st>>>(nx, cand, p.hx, g.rxoff, p.w, g.nz,
                                                             queues, ctr);
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
        const size_t sm = (size_t)8 * W_CAP * sizeof(int32_t);
        tbegin(TM_LIGHT_WARP);
        light_warp_kernel<W_CAP><<<grid_for((int64_t)hc.q[Q_WARP] * 32, 256, 152 * 16), 256, sm, st>>>(
            A, queues + (int64_t)Q_WARP * nx, ctr, Q_WARP);
        JP_CHECK_LAUNCH();
        tend(TM_LIGHT_WARP);
    }
    if (hc.q[Q_W2]) {
        const size_t sm = (size_t)8 * W2_CAP * sizeof(int32_t);   // 64 KB: 3 blocks per SM
        static bool attr2 = false;
        if (!attr2) {
            JP_CUDA_TRY(cudaFuncSetAttribute(light_warp_kernel<W2_CAP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            attr2 = true;
        }
        tbegin(TM_LIGHT_C2);
        light_warp_kernel<W2_CAP><<<grid_for((int64_t)hc.q[Q_W2] * 32, 256, 152 * 3), 256, sm, st>>>(
            A, queues + (int64_t)Q_W2 * nx, ctr, Q_W2);
        JP_CHECK_LAUNCH();
        tend(TM_LIGHT_C2);
    }
    if (hc.q[Q_BITMAP]) {
        int64_t words = (g.nz + 31) / 32;
        int32_t win = (int32_t)std::min<int64_t>(words, BM_MAX_WORDS);
        win = (win + 1023) & ~1023;                 // whole summary words
        const size_t sm = (size_t)(win + win / 32) * sizeof(uint32_t);
        static bool attrb = false;
        if (!attrb) {
            JP_CUDA_TRY(cudaFuncSetAttribute(
                light_bitmap_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                (int)((BM_MAX_WORDS + BM_MAX_WORDS / 32) * sizeof(uint32_t))));
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
