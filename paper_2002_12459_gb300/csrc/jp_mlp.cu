// Learned threshold predictor: degree features and a small MLP trained on the
// GPU.
//
// The paper picks Delta1, Delta2 with a cost model (Section 5, Algorithm 3)
// whose constants it measures by hand (Table 2).  The predictor replaces that
// model by a network trained on thresholds the GPU method itself found best:
//
//  features  two 64-bin log-degree histograms (x degrees; y degrees taken as
//            max(deg_R(y), deg_S(y)), the partition rule); a bin holding c
//            values enters as log2(1 + c) / 32, so the relation's size is
//            visible.  bin(d) = min(63, floor(4 log2 d)) is computed exactly
//            with integers: e = floor(log2 d) from the leading-zero count, and
//            the quarter-octave is found by comparing d * 2^(30 - e) with the
//            ceilings of 2^(30 + k/4), k = 1, 2, 3.
//  network   128 -> 256 -> 256 -> 2, ReLU, output (ln Delta1, ln Delta2).
//            Weights are used in bfloat16, every product and sum in float32;
//            float32 master weights are updated by Adam.
//  kernels   one thread per output element for the forward layers, the input
//            gradients and the weight gradients (the matrices are at most
//            256 x 256 and batches at most 1024, so these simple kernels are
//            far from the query's cost).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "jp_internal.cuh"

struct jp_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    float* master = nullptr;       // [JP_MLP_PARAMS] fp32 master weights
    __nv_bfloat16* w16 = nullptr;  // bf16 copy used by forward/backward
    float* grad = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* act = nullptr;          // activations and gradients for up to MAXB rows
    float* io = nullptr;           // staged X, T, Y
    float* loss = nullptr;
    int64_t step = 0;
};

namespace jp {
namespace {

constexpr int D0 = 128, D1 = 256, D2 = 256, D3 = 2;
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + D0 * D1;
constexpr int OFF_W2 = OFF_B1 + D1;
constexpr int OFF_B2 = OFF_W2 + D1 * D2;
constexpr int OFF_W3 = OFF_B2 + D2;
constexpr int OFF_B3 = OFF_W3 + D2 * D3;
constexpr int NPARAM = OFF_B3 + D3;
constexpr int MAXB = 1024;
static_assert(NPARAM == JP_MLP_PARAMS, "parameter layout");

// activation buffer layout (floats): Z1 H1 Z2 H2 Y dY dH2 dH1 (rows of MAXB)
constexpr size_t A_Z1 = 0, A_H1 = A_Z1 + (size_t)MAXB * D1, A_Z2 = A_H1 + (size_t)MAXB * D1,
                 A_H2 = A_Z2 + (size_t)MAXB * D2, A_Y = A_H2 + (size_t)MAXB * D2,
                 A_DY = A_Y + (size_t)MAXB * D3, A_DH2 = A_DY + (size_t)MAXB * D3,
                 A_DH1 = A_DH2 + (size_t)MAXB * D2, A_TOTAL = A_DH1 + (size_t)MAXB * D1;

// ceilings of 2^(30 + k/4), k = 1, 2, 3
constexpr uint32_t QT1 = 1276901417u, QT2 = 1518500250u, QT3 = 1805811302u;

__device__ __forceinline__ int degree_bin(uint32_t d) {
    const int e = 31 - __clz(d);                 // floor(log2 d), d >= 1
    const uint32_t m = d << (30 - min(e, 30));   // in [2^30, 2^31) for e <= 30
    int b = 4 * e + (m >= QT1) + (m >= QT2) + (m >= QT3);
    return b > 63 ? 63 : b;
}

__global__ void degree_hist_kernel(const int32_t* da, const int32_t* db, int64_t n,
                                   unsigned long long* hist /* [64] */) {
    __shared__ unsigned int h[64];
    if (threadIdx.x < 64) h[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t d = da[i];
        if (db) d = max(d, db[i]);
        if (d >= 1) atomicAdd(&h[degree_bin((uint32_t)d)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 64 && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], (unsigned long long)h[threadIdx.x]);
}

__global__ void to_bf16_kernel(const float* in, __nv_bfloat16* out, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(in[i]);
}

// out[b][j] = act(sum_i in[b][i] * W[i][j] + bias[j]); Z keeps the pre-activation
__global__ void dense_fwd_kernel(const float* in, int B, int din, int dout,
                                 const __nv_bfloat16* W, const __nv_bfloat16* bias, float* Z,
                                 float* out, int relu) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (j >= dout || b >= B) return;
    float s = __bfloat162float(bias[j]);
    const float* x = in + (size_t)b * din;
    for (int i = 0; i < din; ++i) s = fmaf(x[i], __bfloat162float(W[(size_t)i * dout + j]), s);
    if (Z) Z[(size_t)b * dout + j] = s;
    out[(size_t)b * dout + j] = relu ? fmaxf(s, 0.0f) : s;
}

// dY = 2 (Y - T) / B; loss = mean_b ||Y_b - T_b||^2 (single block)
__global__ void mse_grad_kernel(const float* Y, const float* T, int B, float* dY, float* loss) {
    __shared__ float part[256];
    float acc = 0.0f;
    for (int i = threadIdx.x; i < B * D3; i += blockDim.x) {
        const float r = Y[i] - T[i];
        dY[i] = 2.0f * r / (float)B;
        acc += r * r;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = part[0] / (float)B;
}

// dW[i][j] = sum_b in[b][i] * dout[b][j]   (thread per (i, j)); dbias[j] by row i == 0
__global__ void dense_wgrad_kernel(const float* in, const float* dout, int B, int din, int nout,
                                   float* dW, float* dbias) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= nout || i >= din) return;
    float s = 0.0f, sb = 0.0f;
    for (int b = 0; b < B; ++b) {
        const float g = dout[(size_t)b * nout + j];
        s = fmaf(in[(size_t)b * din + i], g, s);
        sb += g;
    }
    dW[(size_t)i * nout + j] = s;
    if (i == 0) dbias[j] = sb;
}

// din_[b][i] = (sum_j dout[b][j] * W[i][j]) * (Z[b][i] > 0)   (thread per (b, i))
__global__ void dense_igrad_kernel(const float* dout, int B, int din, int nout,
                                   const __nv_bfloat16* W, const float* Z, float* din_) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (i >= din || b >= B) return;
    float s = 0.0f;
    for (int j = 0; j < nout; ++j)
        s = fmaf(dout[(size_t)b * nout + j], __bfloat162float(W[(size_t)i * nout + j]), s);
    din_[(size_t)b * din + i] = Z[(size_t)b * din + i] > 0.0f ? s : 0.0f;
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int n, float lr,
                            float b1, float b2, float c1, float c2, float eps) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

void sync_bf16(jp_mlp* M) {
    to_bf16_kernel<<<grid_for(NPARAM, 256, 152 * 4), 256, 0, M->stream>>>(M->master, M->w16, NPARAM);
    JP_CHECK_LAUNCH();
}

// forward of B rows already staged at X (device)
void forward_dev(jp_mlp* M, const float* X, int B) {
    float* a = M->act;
    const __nv_bfloat16* w = M->w16;
    dim3 g1((D1 + 127) / 128, B), g3((D3 + 127) / 128, B);
    dense_fwd_kernel<<<g1, 128, 0, M->stream>>>(X, B, D0, D1, w + OFF_W1, w + OFF_B1, a + A_Z1, a + A_H1, 1);
    JP_CHECK_LAUNCH();
    dense_fwd_kernel<<<g1, 128, 0, M->stream>>>(a + A_H1, B, D1, D2, w + OFF_W2, w + OFF_B2, a + A_Z2, a + A_H2, 1);
    JP_CHECK_LAUNCH();
    dense_fwd_kernel<<<g3, 128, 0, M->stream>>>(a + A_H2, B, D2, D3, w + OFF_W3, w + OFF_B3, nullptr, a + A_Y, 0);
    JP_CHECK_LAUNCH();
}

// gradients of the mean squared error into M->grad
void backward_dev(jp_mlp* M, const float* X, const float* T, int B) {
    float* a = M->act;
    float* gr = M->grad;
    const __nv_bfloat16* w = M->w16;
    mse_grad_kernel<<<1, 256, 0, M->stream>>>(a + A_Y, T, B, a + A_DY, M->loss);
    JP_CHECK_LAUNCH();
    dense_wgrad_kernel<<<dim3((D3 + 127) / 128, D2), 128, 0, M->stream>>>(a + A_H2, a + A_DY, B, D2, D3, gr + OFF_W3, gr + OFF_B3);
    JP_CHECK_LAUNCH();
    dense_igrad_kernel<<<dim3((D2 + 127) / 128, B), 128, 0, M->stream>>>(a + A_DY, B, D2, D3, w + OFF_W3, a + A_Z2, a + A_DH2);
    JP_CHECK_LAUNCH();
    dense_wgrad_kernel<<<dim3((D2 + 127) / 128, D1), 128, 0, M->stream>>>(a + A_H1, a + A_DH2, B, D1, D2, gr + OFF_W2, gr + OFF_B2);
    JP_CHECK_LAUNCH();
    dense_igrad_kernel<<<dim3((D1 + 127) / 128, B), 128, 0, M->stream>>>(a + A_DH2, B, D1, D2, w + OFF_W2, a + A_Z1, a + A_DH1);
    JP_CHECK_LAUNCH();
    dense_wgrad_kernel<<<dim3((D1 + 127) / 128, D0), 128, 0, M->stream>>>(X, a + A_DH1, B, D0, D1, gr + OFF_W1, gr + OFF_B1);
    JP_CHECK_LAUNCH();
}

}  // namespace

// Features of a built graph: x degree histogram and y degree histogram.
void graph_features(const Graph& g, float* host128, Arena& ws, cudaStream_t st) {
    unsigned long long* hist = ws.get<unsigned long long>(128);
    JP_CUDA_TRY(cudaMemsetAsync(hist, 0, 128 * sizeof(unsigned long long), st));
    if (g.nx > 0) {
        degree_hist_kernel<<<grid_for(g.nx, 256, 152 * 4), 256, 0, st>>>(g.deg_rx, nullptr, g.nx, hist);
        JP_CHECK_LAUNCH();
    }
    if (g.ny > 0) {
        degree_hist_kernel<<<grid_for(g.ny, 256, 152 * 4), 256, 0, st>>>(
            g.deg_ry, g.self ? nullptr : g.deg_sy, g.ny, hist + 64);
        JP_CHECK_LAUNCH();
    }
    unsigned long long h[128];
    JP_CUDA_TRY(cudaMemcpyAsync(h, hist, sizeof(h), cudaMemcpyDeviceToHost, st));
    JP_CUDA_TRY(cudaStreamSynchronize(st));
    // a bin holding c values enters as log2(1 + c) / 32 (keeps the scale)
    for (int i = 0; i < 128; ++i) host128[i] = (float)(std::log2(1.0 + (double)h[i]) / 32.0);
}

// Thresholds predicted for the features (ln outputs exponentiated, floored,
// clamped to [1, N]).
void mlp_predict(jp_mlp* M, const float* host128, int64_t N, int64_t* d1, int64_t* d2) {
    JP_CUDA_TRY(cudaMemcpyAsync(M->io, host128, D0 * sizeof(float), cudaMemcpyHostToDevice, M->stream));
    forward_dev(M, M->io, 1);
    float y[2];
    JP_CUDA_TRY(cudaMemcpyAsync(y, M->act + A_Y, sizeof(y), cudaMemcpyDeviceToHost, M->stream));
    JP_CUDA_TRY(cudaStreamSynchronize(M->stream));
    auto conv = [N](float ln) {
        double d = std::exp((double)std::fmin(std::fmax(ln, 0.0f), 40.0f));
        int64_t v = (int64_t)std::floor(d);
        return v < 1 ? (int64_t)1 : (v > N ? N : v);
    };
    *d1 = conv(y[0]);
    *d2 = conv(y[1]);
}

}  // namespace jp

// ------------------------------------------------------------------ C-ABI

extern "C" int jp_mlp_create(jp_mlp** out, int device, void* stream) {
    if (!out) return JP_EINVAL;
    *out = nullptr;
    jp_mlp* M = new (std::nothrow) jp_mlp();
    if (!M) return JP_ENOMEM;
    try {
        JP_CUDA_TRY(cudaSetDevice(device));
        M->device = device;
        M->stream = (cudaStream_t)stream;
        JP_CUDA_TRY(cudaMalloc((void**)&M->master, jp::NPARAM * sizeof(float)));
        JP_CUDA_TRY(cudaMalloc((void**)&M->w16, jp::NPARAM * sizeof(__nv_bfloat16)));
        JP_CUDA_TRY(cudaMalloc((void**)&M->grad, jp::NPARAM * sizeof(float)));
        JP_CUDA_TRY(cudaMalloc((void**)&M->m, jp::NPARAM * sizeof(float)));
        JP_CUDA_TRY(cudaMalloc((void**)&M->v, jp::NPARAM * sizeof(float)));
        JP_CUDA_TRY(cudaMalloc((void**)&M->act, jp::A_TOTAL * sizeof(float)));
        JP_CUDA_TRY(cudaMalloc((void**)&M->io, (size_t)jp::MAXB * (jp::D0 + 2 * jp::D3) * sizeof(float)));
        JP_CUDA_TRY(cudaMalloc((void**)&M->loss, sizeof(float)));
        JP_CUDA_TRY(cudaMemsetAsync(M->master, 0, jp::NPARAM * sizeof(float), M->stream));
        JP_CUDA_TRY(cudaMemsetAsync(M->m, 0, jp::NPARAM * sizeof(float), M->stream));
        JP_CUDA_TRY(cudaMemsetAsync(M->v, 0, jp::NPARAM * sizeof(float), M->stream));
        jp::sync_bf16(M);
        JP_CUDA_TRY(cudaStreamSynchronize(M->stream));
    } catch (const jp::Error& e) {
        jp_mlp_destroy(M);
        return e.code;
    }
    *out = M;
    return JP_OK;
}

extern "C" void jp_mlp_destroy(jp_mlp* M) {
    if (!M) return;
    cudaSetDevice(M->device);
    cudaStreamSynchronize(M->stream);
    cudaFree(M->master);
    cudaFree(M->w16);
    cudaFree(M->grad);
    cudaFree(M->m);
    cudaFree(M->v);
    cudaFree(M->act);
    cudaFree(M->io);
    cudaFree(M->loss);
    cudaGetLastError();
    delete M;
}

extern "C" int jp_mlp_set_params(jp_mlp* M, const float* host, int64_t n) {
    if (!M || !host || n != JP_MLP_PARAMS) return JP_EINVAL;
    try {
        JP_CUDA_TRY(cudaSetDevice(M->device));
        JP_CUDA_TRY(cudaMemcpyAsync(M->master, host, n * sizeof(float), cudaMemcpyHostToDevice, M->stream));
        JP_CUDA_TRY(cudaMemsetAsync(M->m, 0, n * sizeof(float), M->stream));
        JP_CUDA_TRY(cudaMemsetAsync(M->v, 0, n * sizeof(float), M->stream));
        M->step = 0;
        jp::sync_bf16(M);
        JP_CUDA_TRY(cudaStreamSynchronize(M->stream));
    } catch (const jp::Error& e) {
        return e.code;
    }
    return JP_OK;
}

extern "C" int jp_mlp_get_params(jp_mlp* M, float* host, int64_t n) {
    if (!M || !host || n != JP_MLP_PARAMS) return JP_EINVAL;
    try {
        JP_CUDA_TRY(cudaSetDevice(M->device));
        JP_CUDA_TRY(cudaMemcpyAsync(host, M->master, n * sizeof(float), cudaMemcpyDeviceToHost, M->stream));
        JP_CUDA_TRY(cudaStreamSynchronize(M->stream));
    } catch (const jp::Error& e) {
        return e.code;
    }
    return JP_OK;
}

extern "C" int jp_mlp_forward(jp_mlp* M, const float* X, int B, float* Y) {
    if (!M || !X || !Y || B < 1 || B > jp::MAXB) return JP_EINVAL;
    try {
        JP_CUDA_TRY(cudaSetDevice(M->device));
        JP_CUDA_TRY(cudaMemcpyAsync(M->io, X, (size_t)B * jp::D0 * sizeof(float), cudaMemcpyHostToDevice, M->stream));
        jp::forward_dev(M, M->io, B);
        JP_CUDA_TRY(cudaMemcpyAsync(Y, M->act + jp::A_Y, (size_t)B * jp::D3 * sizeof(float), cudaMemcpyDeviceToHost, M->stream));
        JP_CUDA_TRY(cudaStreamSynchronize(M->stream));
    } catch (const jp::Error& e) {
        return e.code;
    }
    return JP_OK;
}

extern "C" int jp_mlp_gradients(jp_mlp* M, const float* X, const float* T, int B, float* grad,
                                float* loss) {
    if (!M || !X || !T || B < 1 || B > jp::MAXB) return JP_EINVAL;
    try {
        JP_CUDA_TRY(cudaSetDevice(M->device));
        float* dX = M->io;
        float* dT = M->io + (size_t)jp::MAXB * jp::D0;
        JP_CUDA_TRY(cudaMemcpyAsync(dX, X, (size_t)B * jp::D0 * sizeof(float), cudaMemcpyHostToDevice, M->stream));
        JP_CUDA_TRY(cudaMemcpyAsync(dT, T, (size_t)B * jp::D3 * sizeof(float), cudaMemcpyHostToDevice, M->stream));
        jp::forward_dev(M, dX, B);
        jp::backward_dev(M, dX, dT, B);
        if (grad)
            JP_CUDA_TRY(cudaMemcpyAsync(grad, M->grad, jp::NPARAM * sizeof(float), cudaMemcpyDeviceToHost, M->stream));
        if (loss) JP_CUDA_TRY(cudaMemcpyAsync(loss, M->loss, sizeof(float), cudaMemcpyDeviceToHost, M->stream));
        JP_CUDA_TRY(cudaStreamSynchronize(M->stream));
    } catch (const jp::Error& e) {
        return e.code;
    }
    return JP_OK;
}

extern "C" int jp_mlp_train_step(jp_mlp* M, const float* X, const float* T, int B, float lr,
                                 float* loss) {
    int rc = jp_mlp_gradients(M, X, T, B, nullptr, loss);
    if (rc) return rc;
    try {
        M->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.0f - std::pow(b1, (float)M->step);
        const float c2 = 1.0f - std::pow(b2, (float)M->step);
        jp::adam_kernel<<<jp::grid_for(jp::NPARAM, 256, 152 * 4), 256, 0, M->stream>>>(
            M->master, M->grad, M->m, M->v, jp::NPARAM, lr, b1, b2, c1, c2, 1e-8f);
        JP_CHECK_LAUNCH();
        jp::sync_bf16(M);
        JP_CUDA_TRY(cudaStreamSynchronize(M->stream));
    } catch (const jp::Error& e) {
        return e.code;
    }
    return JP_OK;
}
