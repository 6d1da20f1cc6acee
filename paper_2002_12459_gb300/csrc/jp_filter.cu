// Boolean set intersection queries in batches (Section 3.3): a set T of
// candidate pairs (x, z) is answered with T ∩ Q, Q(x,z) = R(x,y), S(z,y), i.e.
// the query Q_batch(x,z) = R(x,y), S(z,y), T(x,z).
//
// Only the x values of T can start an answer and only its z values can end
// one, so R is first reduced to the tuples whose x occurs in T and S to those
// whose z occurs in T (semi-joins, as the section's experiments do before
// running Algorithm 1); Q of the reduced relations holds every answer.  Its
// sorted output is then searched for each pair of T.
#include "jp_internal.cuh"

namespace jp {
namespace {

constexpr uint32_t BIAS = 0x80000000u;

inline int G(int64_t n) { return grid_for(n, 256, 152 * 16); }

__global__ void pair_keys_kernel(const int32_t* a, const int32_t* b, int64_t n, uint64_t* keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = ((uint64_t)((uint32_t)a[i] ^ BIAS) << 32) | ((uint32_t)b[i] ^ BIAS);
}

__global__ void one_key_kernel(const int32_t* a, int64_t n, uint64_t* keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = (uint32_t)a[i] ^ BIAS;
}

__device__ __forceinline__ bool contains(const uint64_t* dict, int64_t n, uint64_t k) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (dict[mid] < k) lo = mid + 1; else hi = mid;
    }
    return lo < n && dict[lo] == k;
}

// flag[i] = 1 iff col[i] is one of the sorted distinct (biased) values in dict
__global__ void member_kernel(const int32_t* col, int64_t n, const uint64_t* dict, int64_t nd,
                              uint32_t* flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = contains(dict, nd, (uint32_t)col[i] ^ BIAS) ? 1u : 0u;
}

__global__ void compact2_kernel(const int32_t* a, const int32_t* b, int64_t n, const uint32_t* flag,
                                const uint32_t* pos, int32_t* oa, int32_t* ob) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) {
            oa[pos[i]] = a[i];
            ob[pos[i]] = b[i];
        }
}

// flag[i] = 1 iff pair i of T (biased key) is one of the sorted output pairs
__global__ void found_kernel(const uint64_t* tkeys, int64_t nt, const int32_t* ox, const int32_t* oz,
                             int64_t no, uint32_t* flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nt;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = tkeys[i];
        int64_t lo = 0, hi = no;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            const uint64_t m = ((uint64_t)((uint32_t)ox[mid] ^ BIAS) << 32) | ((uint32_t)oz[mid] ^ BIAS);
            if (m < k) lo = mid + 1; else hi = mid;
        }
        flag[i] = (lo < no && ox[lo] == (int32_t)((uint32_t)(k >> 32) ^ BIAS) &&
                   oz[lo] == (int32_t)((uint32_t)k ^ BIAS)) ? 1u : 0u;
    }
}

__global__ void emit_pairs_kernel(const uint64_t* tkeys, int64_t nt, const uint32_t* flag,
                                  const uint32_t* pos, int32_t* ox, int32_t* oz) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nt;
         i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) {
            ox[pos[i]] = (int32_t)((uint32_t)(tkeys[i] >> 32) ^ BIAS);
            oz[pos[i]] = (int32_t)((uint32_t)tkeys[i] ^ BIAS);
        }
}

uint32_t read_count(const uint32_t* d, cudaStream_t st) {
    uint32_t v = 0;
    JP_CUDA_TRY(cudaMemcpyAsync(&v, d, sizeof(v), cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaStreamSynchronize(st));
    return v;
}

// sorted distinct keys of keys[0..n) (keys and tmp are scratch)
uint64_t* distinct(uint64_t* keys, uint64_t* tmp, int64_t n, int64_t* count, Arena& ws,
                   cudaStream_t st, uint32_t* hist_host) {
    uint64_t* s = radix_sort_u64(keys, tmp, n, ws, st, hist_host);
    uint64_t* u = (s == keys) ? tmp : keys;
    uint32_t* d = ws.get<uint32_t>(1);
    unique_u64(s, n, u, d, ws, st);
    *count = read_count(d, st);
    return u;
}

// the tuples of (a, b) whose a is one of dict's values
jp_rel keep_members(const int32_t* a, const int32_t* b, int64_t n, const uint64_t* dict, int64_t nd,
                    Arena& ws, cudaStream_t st) {
    uint32_t* flag = ws.get<uint32_t>(n + 1);
    uint32_t* pos = ws.get<uint32_t>(n + 1);
    uint32_t* d = ws.get<uint32_t>(1);
    if (n > 0) {
        member_kernel<<<G(n), 256, 0, st>>>(a, n, dict, nd, flag);
        JP_CHECK_LAUNCH();
    }
    scan_u32(flag, pos, n, d, ws, st);
    const int64_t m = n > 0 ? read_count(d, st) : 0;
    jp_rel r;
    int32_t* oa = ws.get<int32_t>(m + 1);
    int32_t* ob = ws.get<int32_t>(m + 1);
    if (n > 0) {
        compact2_kernel<<<G(n), 256, 0, st>>>(a, b, n, flag, pos, oa, ob);
        JP_CHECK_LAUNCH();
    }
    r.x = oa;
    r.y = ob;
    r.n = m;
    return r;
}

}  // namespace

void filter_reduce(const jp_rel& R, const jp_rel& S, const jp_rel& T, FilterState& fs, Arena& ws,
                   cudaStream_t st, uint32_t* hist_host) {
    const int64_t nt = T.n;
    const int64_t m = nt > 0 ? nt : 1;
    uint64_t* k0 = ws.get<uint64_t>(m);
    uint64_t* k1 = ws.get<uint64_t>(m);
    if (nt > 0) {
        pair_keys_kernel<<<G(nt), 256, 0, st>>>(T.x, T.y, nt, k0);
        JP_CHECK_LAUNCH();
    }
    fs.tkeys = distinct(k0, k1, nt, &fs.nt, ws, st, hist_host);
    // the distinct x and the distinct z values of T
    uint64_t* v0 = ws.get<uint64_t>(m);
    uint64_t* v1 = ws.get<uint64_t>(m);
    if (nt > 0) {
        one_key_kernel<<<G(nt), 256, 0, st>>>(T.x, nt, v0);
        JP_CHECK_LAUNCH();
    }
    int64_t nx = 0, nz = 0;
    const uint64_t* xs = distinct(v0, v1, nt, &nx, ws, st, hist_host);
    uint64_t* w0 = ws.get<uint64_t>(m);
    uint64_t* w1 = ws.get<uint64_t>(m);
    if (nt > 0) {
        one_key_kernel<<<G(nt), 256, 0, st>>>(T.y, nt, w0);
        JP_CHECK_LAUNCH();
    }
    const uint64_t* zs = distinct(w0, w1, nt, &nz, ws, st, hist_host);
    fs.R = keep_members(R.x, R.y, R.n, xs, nx, ws, st);
    fs.S = keep_members(S.x, S.y, S.n, zs, nz, ws, st);
}

int64_t filter_find(FilterState& fs, const int32_t* ox, const int32_t* oz, int64_t no, Arena& ws,
                    cudaStream_t st) {
    const int64_t nt = fs.nt;
    fs.flag = ws.get<uint32_t>(nt + 1);
    fs.pos = ws.get<uint32_t>(nt + 1);
    uint32_t* d = ws.get<uint32_t>(1);
    if (nt > 0) {
        found_kernel<<<G(nt), 256, 0, st>>>(fs.tkeys, nt, ox, oz, no, fs.flag);
        JP_CHECK_LAUNCH();
    }
    scan_u32(fs.flag, fs.pos, nt, d, ws, st);
    return nt > 0 ? read_count(d, st) : 0;
}

void filter_emit(const FilterState& fs, int32_t* px, int32_t* pz, cudaStream_t st) {
    if (fs.nt <= 0) return;
    emit_pairs_kernel<<<G(fs.nt), 256, 0, st>>>(fs.tkeys, fs.nt, fs.flag, fs.pos, px, pz);
    JP_CHECK_LAUNCH();
}

}  // namespace jp
