// Batches of two-path queries evaluated in one pass of the pipeline.
//
// A batch of self-joins Q_q(x,z) = R_q(x,y), R_q(z,y), q = 0..nq-1, is the
// single self-join of the disjoint union of the R_q once every value carries
// its query: (q, x) and (q, y) are dictionary-encoded to global ids in
// (q, value) order, so the x ids of query q form one contiguous range, and no
// y id is shared by two queries, so no witness joins tuples of two queries.
// The union then runs through the same passes as one query (each pass one
// launch for the whole batch, its work spread over all queries' rows); its
// sorted output is the queries' sorted outputs one after another, mapped back
// to values at placement, and query q's pairs start at the output offset of
// its first x id.
#include "jp_internal.cuh"

namespace jp {
namespace {

constexpr uint32_t BIAS = 0x80000000u;

inline int G(int64_t n) { return grid_for(n, 256, 152 * 16); }

// key of tuple i: (q << 32) | biased value, q found in the query offsets
__global__ void tag_kernel(const int32_t* __restrict__ x, const int32_t* __restrict__ y, int64_t n,
                           const int64_t* __restrict__ qoff, int32_t nq, uint64_t* kx,
                           uint64_t* ky) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = nq;            // last q with qoff[q] <= i
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (qoff[mid] <= i) lo = mid; else hi = mid;
        }
        const uint64_t q = (uint64_t)lo << 32;
        kx[i] = q | ((uint32_t)x[i] ^ BIAS);
        ky[i] = q | ((uint32_t)y[i] ^ BIAS);
    }
}

// id of every key in the sorted distinct keys (each key is present)
__global__ void find_kernel(const uint64_t* __restrict__ dict, int64_t nd,
                            const uint64_t* __restrict__ keys, int64_t n, int32_t* __restrict__ id,
                            uint32_t* status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        int64_t lo = 0, hi = nd;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (dict[mid] < k) lo = mid + 1; else hi = mid;
        }
        if (lo >= nd || dict[lo] != k) {
            atomicOr(status, ST_BADINDEX);
            lo = 0;
        }
        id[i] = (int32_t)lo;
    }
}

__global__ void value_kernel(const uint64_t* __restrict__ dict, int64_t nd, int32_t* __restrict__ val) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nd;
         i += (int64_t)gridDim.x * blockDim.x)
        val[i] = (int32_t)((uint32_t)dict[i] ^ BIAS);
}

// first x id of every query: lower bound of (q << 32) in the distinct x keys
__global__ void query_begin_kernel(const uint64_t* __restrict__ dict, int64_t nd, int32_t nq,
                                   int32_t* __restrict__ begin) {
    for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q <= nq; q += gridDim.x * blockDim.x) {
        const uint64_t k = (uint64_t)q << 32;
        int64_t lo = 0, hi = nd;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (dict[mid] < k) lo = mid + 1; else hi = mid;
        }
        begin[q] = (int32_t)lo;
    }
}

__global__ void gather_off_kernel(const int64_t* __restrict__ out_off, int64_t nx, int64_t count,
                                  const int32_t* __restrict__ begin, int32_t nq,
                                  int64_t* __restrict__ off) {
    for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q <= nq; q += gridDim.x * blockDim.x) {
        const int64_t b = begin[q];
        off[q] = b < nx ? out_off[b] : count;
    }
}

uint64_t* sorted_distinct(uint64_t* keys, uint64_t* tmp, int64_t n, int64_t* count, Arena& ws,
                          cudaStream_t st, uint32_t* hist_host) {
    uint64_t* sorted = radix_sort_u64(keys, tmp, n, ws, st, hist_host);
    uint64_t* out = (sorted == keys) ? tmp : keys;
    uint32_t* d_cnt = ws.get<uint32_t>(1);
    unique_u64(sorted, n, out, d_cnt, ws, st);
    uint32_t c = 0;
    JP_CUDA_TRY(cudaMemcpyAsync(&c, d_cnt, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaStreamSynchronize(st));
    *count = c;
    return out;
}

}  // namespace

void batch_encode(const int32_t* x, const int32_t* y, int64_t n, int32_t nq,
                  const int64_t* qoff_host, BatchIds& b, Arena& ws, cudaStream_t st,
                  uint32_t* hist_host, uint32_t* d_status) {
    int64_t* qoff = ws.get<int64_t>((size_t)nq + 1);
    JP_CUDA_TRY(cudaMemcpyAsync(qoff, qoff_host, ((size_t)nq + 1) * sizeof(int64_t),
                                cudaMemcpyHostToDevice, st));
    const int64_t m = n > 0 ? n : 1;
    uint64_t* kx = ws.get<uint64_t>(m);
    uint64_t* ky = ws.get<uint64_t>(m);
    uint64_t* t0 = ws.get<uint64_t>(m);
    uint64_t* t1 = ws.get<uint64_t>(m);
    b.xg = ws.get<int32_t>(m);
    b.yg = ws.get<int32_t>(m);
    b.xq_begin = ws.get<int32_t>((size_t)nq + 1);
    b.yq_begin = ws.get<int32_t>((size_t)nq + 1);
    if (n > 0) {
        tag_kernel<<<G(n), 256, 0, st>>>(x, y, n, qoff, nq, kx, ky);
        JP_CHECK_LAUNCH();
        // x: sorted distinct (q, x) -> ids, values, query ranges
        JP_CUDA_TRY(cudaMemcpyAsync(t0, kx, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
        int64_t nxg = 0;
        uint64_t* ux = sorted_distinct(t0, t1, n, &nxg, ws, st, hist_host);
        b.nxg = nxg;
        b.xorig = ws.get<int32_t>(nxg + 1);
        value_kernel<<<G(nxg), 256, 0, st>>>(ux, nxg, b.xorig);
        JP_CHECK_LAUNCH();
        find_kernel<<<G(n), 256, 0, st>>>(ux, nxg, kx, n, b.xg, d_status);
        JP_CHECK_LAUNCH();
        query_begin_kernel<<<grid_for((int64_t)nq + 1, 256, 152), 256, 0, st>>>(ux, nxg, nq,
                                                                                b.xq_begin);
        JP_CHECK_LAUNCH();
        // y: sorted distinct (q, y) -> ids (only their identity matters)
        uint64_t* u0 = ws.get<uint64_t>(m);
        int64_t nyg = 0;
        uint64_t* uy = sorted_distinct(ky, u0, n, &nyg, ws, st, hist_host);
        query_begin_kernel<<<grid_for((int64_t)nq + 1, 256, 152), 256, 0, st>>>(uy, nyg, nq,
                                                                                b.yq_begin);
        JP_CHECK_LAUNCH();
        // ky may now hold scratch: search the distinct keys with a fresh tag pass
        uint64_t* ky2 = (uy == ky) ? u0 : ky;
        tag_kernel<<<G(n), 256, 0, st>>>(x, y, n, qoff, nq, t1, ky2);
        JP_CHECK_LAUNCH();
        find_kernel<<<G(n), 256, 0, st>>>(uy, nyg, ky2, n, b.yg, d_status);
        JP_CHECK_LAUNCH();
    } else {
        b.nxg = 0;
        b.xorig = ws.get<int32_t>(1);
        JP_CUDA_TRY(cudaMemsetAsync(b.xq_begin, 0, ((size_t)nq + 1) * sizeof(int32_t), st));
        JP_CUDA_TRY(cudaMemsetAsync(b.yq_begin, 0, ((size_t)nq + 1) * sizeof(int32_t), st));
    }
}

// ------------------------------------------------------------ star batches
// nq star queries Q*_3 over (R1_q, R2_q, R3_q): relation i holds the queries'
// tuples one after another (qoff_i).  Every x_i and every y is tagged with its
// query and dictionary-encoded: x_i per relation, y over the three relations
// together, so that the three relations of one query share their y ids and no
// two queries share any.  Q*_3 of the tagged union is then the union of the
// queries' answers, each x1 id range holding one query.
namespace {

__global__ void tag_one_kernel(const int32_t* __restrict__ v, int64_t n,
                               const int64_t* __restrict__ qoff, int32_t nq, uint64_t* key) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = nq;            // last q with qoff[q] <= i
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (qoff[mid] <= i) lo = mid; else hi = mid;
        }
        key[i] = ((uint64_t)lo << 32) | ((uint32_t)v[i] ^ BIAS);
    }
}

// first output position whose x1 id is at least begin[q] (the output is
// sorted by x1 id first)
__global__ void star_offsets_kernel(const int32_t* __restrict__ col0, int64_t count,
                                    const int32_t* __restrict__ begin, int32_t nq,
                                    int64_t* __restrict__ off) {
    for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q <= nq; q += gridDim.x * blockDim.x) {
        const int32_t b = begin[q];
        int64_t lo = 0, hi = count;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (col0[mid] < b) lo = mid + 1; else hi = mid;
        }
        off[q] = lo;
    }
}

__global__ void map_cols_kernel(int32_t* c0, int32_t* c1, int32_t* c2, int64_t n,
                                const int32_t* __restrict__ v0, const int32_t* __restrict__ v1,
                                const int32_t* __restrict__ v2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        c0[i] = v0[c0[i]];
        c1[i] = v1[c1[i]];
        c2[i] = v2[c2[i]];
    }
}

}  // namespace

void star_batch_encode(const jp_rel* rels, int32_t nq, const int64_t* qoff_host, StarBatchIds& b,
                       Arena& ws, cudaStream_t st, uint32_t* hist_host, uint32_t* d_status) {
    int64_t* qoff[3];
    int64_t ntot = 0;
    for (int i = 0; i < 3; ++i) {
        qoff[i] = ws.get<int64_t>((size_t)nq + 1);
        JP_CUDA_TRY(cudaMemcpyAsync(qoff[i], qoff_host + (size_t)i * (nq + 1),
                                    ((size_t)nq + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        ntot += rels[i].n;
    }
    // y: the three relations' tagged y together
    const int64_t m = ntot > 0 ? ntot : 1;
    uint64_t* ky = ws.get<uint64_t>(m);
    uint64_t* t0 = ws.get<uint64_t>(m);
    uint64_t* t1 = ws.get<uint64_t>(m);
    int64_t at = 0;
    for (int i = 0; i < 3; ++i) {
        if (rels[i].n > 0) {
            tag_one_kernel<<<G(rels[i].n), 256, 0, st>>>(rels[i].y, rels[i].n, qoff[i], nq, ky + at);
            JP_CHECK_LAUNCH();
        }
        at += rels[i].n;
    }
    if (ntot > 0)
        JP_CUDA_TRY(cudaMemcpyAsync(t0, ky, ntot * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    int64_t nyg = 0;
    uint64_t* uy = sorted_distinct(t0, t1, ntot, &nyg, ws, st, hist_host);
    uint64_t* kx = (uy == t0) ? t1 : t0;      // free buffer for the x keys
    at = 0;
    for (int i = 0; i < 3; ++i) {
        const int64_t n = rels[i].n;
        b.rel[i].n = n;
        int32_t* yg = ws.get<int32_t>(n > 0 ? n : 1);
        int32_t* xg = ws.get<int32_t>(n > 0 ? n : 1);
        if (n > 0) {
            find_kernel<<<G(n), 256, 0, st>>>(uy, nyg, ky + at, n, yg, d_status);
            JP_CHECK_LAUNCH();
            tag_one_kernel<<<G(n), 256, 0, st>>>(rels[i].x, n, qoff[i], nq, kx);
            JP_CHECK_LAUNCH();
        }
        // x_i: sorted distinct tagged values -> ids and values
        uint64_t* s0 = ws.get<uint64_t>(n > 0 ? n : 1);
        uint64_t* s1 = ws.get<uint64_t>(n > 0 ? n : 1);
        if (n > 0)
            JP_CUDA_TRY(cudaMemcpyAsync(s0, kx, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
        int64_t nxg = 0;
        uint64_t* ux = sorted_distinct(s0, s1, n, &nxg, ws, st, hist_host);
        b.xorig[i] = ws.get<int32_t>(nxg + 1);
        if (nxg > 0) {
            value_kernel<<<G(nxg), 256, 0, st>>>(ux, nxg, b.xorig[i]);
            JP_CHECK_LAUNCH();
        }
        if (n > 0) {
            find_kernel<<<G(n), 256, 0, st>>>(ux, nxg, kx, n, xg, d_status);
            JP_CHECK_LAUNCH();
        }
        if (i == 0) {
            b.x1q_begin = ws.get<int32_t>((size_t)nq + 1);
            query_begin_kernel<<<grid_for((int64_t)nq + 1, 256, 152), 256, 0, st>>>(ux, nxg, nq,
                                                                                    b.x1q_begin);
            JP_CHECK_LAUNCH();
        }
        b.rel[i].x = xg;
        b.rel[i].y = yg;
        at += n;
    }
}

void star_batch_finish(int32_t* const* cols, int64_t count, const StarBatchIds& b, int32_t nq,
                       int64_t* host_offsets, Arena& ws, cudaStream_t st) {
    int64_t* off = ws.get<int64_t>((size_t)nq + 1);
    star_offsets_kernel<<<grid_for((int64_t)nq + 1, 256, 152), 256, 0, st>>>(cols[0], count,
                                                                             b.x1q_begin, nq, off);
    JP_CHECK_LAUNCH();
    if (count > 0) {
        map_cols_kernel<<<G(count), 256, 0, st>>>(cols[0], cols[1], cols[2], count, b.xorig[0],
                                                  b.xorig[1], b.xorig[2]);
        JP_CHECK_LAUNCH();
    }
    JP_CUDA_TRY(cudaMemcpyAsync(host_offsets, off, ((size_t)nq + 1) * sizeof(int64_t),
                                cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaStreamSynchronize(st));
}

void batch_offsets(const int64_t* out_off, int64_t nx, int64_t count, const BatchIds& b,
                   int32_t nq, int64_t* host_offsets, Arena& ws, cudaStream_t st) {
    int64_t* off = ws.get<int64_t>((size_t)nq + 1);
    gather_off_kernel<<<grid_for((int64_t)nq + 1, 256, 152), 256, 0, st>>>(out_off, nx, count,
                                                                           b.xq_begin, nq, off);
    JP_CHECK_LAUNCH();
    JP_CUDA_TRY(cudaMemcpyAsync(host_offsets, off, ((size_t)nq + 1) * sizeof(int64_t),
                                cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaStreamSynchronize(st));
}

}  // namespace jp
