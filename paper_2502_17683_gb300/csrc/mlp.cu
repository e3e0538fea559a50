// Learned step proposer for ALS extrapolation: a 40-64-64-1 tanh network,
// alpha = 1 + 3 sigmoid(z) in [1, 4]. Parameters are FP32 master weights; the forward and
// backward kernels round every weight to BF16 when they use it and accumulate in FP32.
// Parameter order: W1 (64 x 40), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3 (1).
// All reductions run in a fixed order, so training is deterministic.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "prof.cuh"
#include "thc_cpd.h"

namespace thc {
namespace {

constexpr int NIN = 40, NH = 64;
constexpr int OW1 = 0, OB1 = OW1 + NH * NIN, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH, NPARAM = OB3 + 1;
static_assert(NPARAM == 6849, "parameter count");

__device__ __forceinline__ float bfw(float w) { return __bfloat162float(__float2bfloat16_rn(w)); }

// forward of sample blockIdx.x (64 threads, one per hidden unit); optional saves
__global__ void __launch_bounds__(NH)
k_mlp_fwd(const float* __restrict__ P, const float* __restrict__ X, const int* __restrict__ idx,
          int n, float* __restrict__ alpha, float* __restrict__ h1s, float* __restrict__ h2s,
          float* __restrict__ ss) {
    const int b = blockIdx.x;
    if (b >= n) return;
    const int row = idx ? idx[b] : b;
    __shared__ float x[NIN], h1[NH], h2[NH], red[NH];
    const int u = threadIdx.x;
    if (u < NIN) x[u] = X[(size_t)row * NIN + u];
    __syncthreads();
    float a = P[OB1 + u];
    for (int i = 0; i < NIN; ++i) a = fmaf(bfw(P[OW1 + u * NIN + i]), x[i], a);
    h1[u] = tanhf(a);
    __syncthreads();
    a = P[OB2 + u];
    for (int j = 0; j < NH; ++j) a = fmaf(bfw(P[OW2 + u * NH + j]), h1[j], a);
    h2[u] = tanhf(a);
    red[u] = bfw(P[OW3 + u]) * h2[u];
    __syncthreads();
    for (int o = NH / 2; o > 0; o >>= 1) {
        if (u < o) red[u] += red[u + o];
        __syncthreads();
    }
    if (u == 0) {
        const float z = red[0] + P[OB3];
        const float s = 1.0f / (1.0f + expf(-z));
        alpha[b] = 1.0f + 3.0f * s;
        if (ss) ss[b] = s;
    }
    if (h1s) h1s[(size_t)b * NH + u] = h1[u];
    if (h2s) h2s[(size_t)b * NH + u] = h2[u];
}

// per-sample deltas of the MSE loss (1/n) sum (alpha - y)^2
__global__ void __launch_bounds__(NH)
k_mlp_delta(const float* __restrict__ P, const float* __restrict__ y, const int* __restrict__ idx,
            int n, const float* __restrict__ alpha, const float* __restrict__ ss,
            const float* __restrict__ h1s, const float* __restrict__ h2s, float* __restrict__ dz,
            float* __restrict__ da1, float* __restrict__ da2) {
    const int b = blockIdx.x;
    if (b >= n) return;
    const int row = idx ? idx[b] : b;
    const int u = threadIdx.x;
    __shared__ float d2[NH];
    const float s = ss[b];
    const float g = 2.0f * (alpha[b] - y[row]) / (float)n * 3.0f * s * (1.0f - s);
    const float h2 = h2s[(size_t)b * NH + u];
    d2[u] = g * bfw(P[OW3 + u]) * (1.0f - h2 * h2);
    __syncthreads();
    float a = 0.0f;
    for (int v = 0; v < NH; ++v) a = fmaf(d2[v], bfw(P[OW2 + v * NH + u]), a);
    const float h1 = h1s[(size_t)b * NH + u];
    da1[(size_t)b * NH + u] = a * (1.0f - h1 * h1);
    da2[(size_t)b * NH + u] = d2[u];
    if (u == 0) dz[b] = g;
}

// gradient of every parameter: sum over the batch in sample order (one thread each)
__global__ void k_mlp_wgrad(const float* __restrict__ X, const int* __restrict__ idx, int n,
                            const float* __restrict__ h1s, const float* __restrict__ h2s,
                            const float* __restrict__ dz, const float* __restrict__ da1,
                            const float* __restrict__ da2, float* __restrict__ G) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    float s = 0.0f;
    if (p < OB1) {
        const int u = p / NIN, i = p % NIN;
        for (int b = 0; b < n; ++b) {
            const int row = idx ? idx[b] : b;
            s = fmaf(da1[(size_t)b * NH + u], X[(size_t)row * NIN + i], s);
        }
    } else if (p < OW2) {
        const int u = p - OB1;
        for (int b = 0; b < n; ++b) s += da1[(size_t)b * NH + u];
    } else if (p < OB2) {
        const int u = (p - OW2) / NH, j = (p - OW2) % NH;
        for (int b = 0; b < n; ++b) s = fmaf(da2[(size_t)b * NH + u], h1s[(size_t)b * NH + j], s);
    } else if (p < OW3) {
        const int u = p - OB2;
        for (int b = 0; b < n; ++b) s += da2[(size_t)b * NH + u];
    } else if (p < OB3) {
        const int u = p - OW3;
        for (int b = 0; b < n; ++b) s = fmaf(dz[b], h2s[(size_t)b * NH + u], s);
    } else {
        for (int b = 0; b < n; ++b) s += dz[b];
    }
    G[p] = s;
}

// loss (1/n) sum (alpha - y)^2, one block, fixed order
__global__ void k_mlp_loss(const float* __restrict__ alpha, const float* __restrict__ y,
                           const int* __restrict__ idx, int n, float* __restrict__ out) {
    __shared__ float sh[256];
    float s = 0.0f;
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        const float r = alpha[b] - y[idx ? idx[b] : b];
        s = fmaf(r, r, s);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] / (float)n;
}

// Adam (Kingma & Ba) with bias correction
__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m,
                       float* __restrict__ v, int t, float lr) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float g = G[p];
    const float mm = b1 * m[p] + (1.0f - b1) * g;
    const float vv = b2 * v[p] + (1.0f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float mh = mm / (1.0f - powf(b1, (float)t));
    const float vh = vv / (1.0f - powf(b2, (float)t));
    P[p] -= lr * mh / (sqrtf(vh) + eps);
}

// SplitMix64 (Steele, Lea & Flood 2014): counter-based uniform numbers for the init
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Glorot-uniform weights, zero biases
__global__ void k_mlp_init(float* __restrict__ P, unsigned long long seed) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    float lim = 0.0f;
    if (p < OB1) lim = sqrtf(6.0f / (NIN + NH));
    else if (p >= OW2 && p < OB2) lim = sqrtf(6.0f / (NH + NH));
    else if (p >= OW3 && p < OB3) lim = sqrtf(6.0f / (NH + 1));
    const unsigned long long r = splitmix64(seed * 0x100000001B3ull + (unsigned long long)p);
    const float u = (float)((r >> 40) * (1.0 / 16777216.0));  // [0, 1)
    P[p] = lim * (2.0f * u - 1.0f);
}

struct MlpWs {
    float *alpha, *s, *h1, *h2, *dz, *da1, *da2, *G, *m, *v, *loss;
    int* idx;
    void* block = nullptr;
    cudaStream_t st;
    ~MlpWs() {
        if (block) cudaFreeAsync(block, st);
    }
};

cudaError_t mlp_ws(MlpWs& w, cudaStream_t st, int nmax) {
    w.st = st;
    Arena a;
    size_t bytes = 0;
    bytes += 4 * Arena::need<float>(nmax) + 4 * Arena::need<float>((size_t)nmax * NH);
    bytes += 3 * Arena::need<float>(NPARAM) + Arena::need<float>(1) + Arena::need<int>(nmax);
    cudaError_t e = cudaMallocAsync(&w.block, bytes, st);
    if (e != cudaSuccess) return e;
    a.base = (char*)w.block;
    w.alpha = a.take<float>(nmax);
    w.s = a.take<float>(nmax);
    w.dz = a.take<float>(nmax);
    w.loss = a.take<float>(1);
    w.h1 = a.take<float>((size_t)nmax * NH);
    w.h2 = a.take<float>((size_t)nmax * NH);
    w.da1 = a.take<float>((size_t)nmax * NH);
    w.da2 = a.take<float>((size_t)nmax * NH);
    w.G = a.take<float>(NPARAM);
    w.m = a.take<float>(NPARAM);
    w.v = a.take<float>(NPARAM);
    w.idx = a.take<int>(nmax);
    (void)a.take<float>(nmax);
    return cudaSuccess;
}

void grad_step(MlpWs& w, const float* P, const float* X, const float* y, const int* idx, int n) {
    k_mlp_fwd<<<n, NH, 0, w.st>>>(P, X, idx, n, w.alpha, w.h1, w.h2, w.s);
    k_mlp_delta<<<n, NH, 0, w.st>>>(P, y, idx, n, w.alpha, w.s, w.h1, w.h2, w.dz, w.da1, w.da2);
    k_mlp_wgrad<<<cdiv(NPARAM, 128), 128, 0, w.st>>>(X, idx, n, w.h1, w.h2, w.dz, w.da1, w.da2, w.G);
    count_launch(3);
}

}  // namespace

// used by the ALS driver: alpha for one feature vector (device in, device out)
void mlp_forward1(cudaStream_t st, const float* P, const float* x, float* alpha) {
    k_mlp_fwd<<<1, NH, 0, st>>>(P, x, nullptr, 1, alpha, nullptr, nullptr, nullptr);
    count_launch();
}

}  // namespace thc

using namespace thc;

static thc_cpd_status mlp_err(thc_cpd_status s, const char* m) { return (thc_cpd_status)set_error(s, m); }

extern "C" thc_cpd_status thc_cpd_mlp_init(float* params, unsigned long long seed,
                                           const thc_cpd_opts* opts) {
    if (!params) return mlp_err(THC_CPD_ERR_ARG, "params must be non-null");
    cudaStream_t st = opts ? (cudaStream_t)opts->stream : (cudaStream_t)0;
    k_mlp_init<<<cdiv(NPARAM, 128), 128, 0, st>>>(params, seed);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? THC_CPD_OK : mlp_err(THC_CPD_ERR_CUDA, "launch failed");
}

extern "C" thc_cpd_status thc_cpd_mlp_forward(const float* params, const float* X, int n,
                                              float* alpha, const thc_cpd_opts* opts) {
    if (!params || !X || !alpha) return mlp_err(THC_CPD_ERR_ARG, "null pointer");
    if (n < 1 || n > (1 << 24)) return mlp_err(THC_CPD_ERR_SHAPE, "n must be in [1, 2^24]");
    cudaStream_t st = opts ? (cudaStream_t)opts->stream : (cudaStream_t)0;
    k_mlp_fwd<<<n, NH, 0, st>>>(params, X, nullptr, n, alpha, nullptr, nullptr, nullptr);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return mlp_err(THC_CPD_ERR_CUDA, "launch failed");
    return cudaStreamSynchronize(st) == cudaSuccess ? THC_CPD_OK : mlp_err(THC_CPD_ERR_CUDA, "sync failed");
}

extern "C" thc_cpd_status thc_cpd_mlp_grad(const float* params, const float* X, const float* y,
                                           int n, float* grad, float* loss_host,
                                           const thc_cpd_opts* opts) {
    if (!params || !X || !y || !grad) return mlp_err(THC_CPD_ERR_ARG, "null pointer");
    if (n < 1 || n > (1 << 20)) return mlp_err(THC_CPD_ERR_SHAPE, "n must be in [1, 2^20]");
    cudaStream_t st = opts ? (cudaStream_t)opts->stream : (cudaStream_t)0;
    MlpWs w;
    if (mlp_ws(w, st, n) != cudaSuccess) return mlp_err(THC_CPD_ERR_ALLOC, "workspace allocation failed");
    grad_step(w, params, X, y, nullptr, n);
    k_mlp_loss<<<1, 256, 0, st>>>(w.alpha, y, nullptr, n, w.loss);
    count_launch();
    cudaMemcpyAsync(grad, w.G, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, st);
    float l = 0.f;
    cudaMemcpyAsync(&l, w.loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return mlp_err(THC_CPD_ERR_CUDA, "gradient failed");
    if (loss_host) *loss_host = l;
    return THC_CPD_OK;
}

extern "C" thc_cpd_status thc_cpd_mlp_adam(float* params, const float* grad, float* m, float* v,
                                           int t, float lr, const thc_cpd_opts* opts) {
    if (!params || !grad || !m || !v) return mlp_err(THC_CPD_ERR_ARG, "null pointer");
    if (t < 1) return mlp_err(THC_CPD_ERR_ARG, "the step count t must be >= 1");
    cudaStream_t st = opts ? (cudaStream_t)opts->stream : (cudaStream_t)0;
    k_adam<<<cdiv(NPARAM, 128), 128, 0, st>>>(params, grad, m, v, t, lr);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return mlp_err(THC_CPD_ERR_CUDA, "launch failed");
    return cudaStreamSynchronize(st) == cudaSuccess ? THC_CPD_OK : mlp_err(THC_CPD_ERR_CUDA, "sync failed");
}

extern "C" thc_cpd_status thc_cpd_mlp_train(float* params, const float* X, const float* y, int n,
                                            int epochs, int batch, float lr,
                                            unsigned long long seed, float* final_loss_host,
                                            const thc_cpd_opts* opts) {
    if (!params || !X || !y) return mlp_err(THC_CPD_ERR_ARG, "null pointer");
    if (n < 1 || batch < 1 || epochs < 0 || n > (1 << 24))
        return mlp_err(THC_CPD_ERR_SHAPE, "bad n / batch / epochs");
    batch = std::min(batch, n);
    cudaStream_t st = opts ? (cudaStream_t)opts->stream : (cudaStream_t)0;
    MlpWs w;
    if (mlp_ws(w, st, std::max(n, batch)) != cudaSuccess)
        return mlp_err(THC_CPD_ERR_ALLOC, "workspace allocation failed");
    cudaMemsetAsync(w.m, 0, sizeof(float) * NPARAM, st);
    cudaMemsetAsync(w.v, 0, sizeof(float) * NPARAM, st);
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    int* dperm = nullptr;
    if (cudaMallocAsync((void**)&dperm, sizeof(int) * n, st) != cudaSuccess)
        return mlp_err(THC_CPD_ERR_ALLOC, "workspace allocation failed");
    unsigned long long rs = seed ^ 0xA5A5A5A5ull;
    auto rnd = [&]() {  // SplitMix64 on the host for the epoch shuffles
        rs += 0x9E3779B97F4A7C15ull;
        unsigned long long z = rs;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    int t = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int i = n - 1; i > 0; --i) std::swap(perm[i], perm[(int)(rnd() % (unsigned long long)(i + 1))]);
        cudaMemcpyAsync(dperm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
        cudaStreamSynchronize(st);  // perm is reused next epoch
        for (int b0 = 0; b0 + batch <= n; b0 += batch) {
            grad_step(w, params, X, y, dperm + b0, batch);
            k_adam<<<cdiv(NPARAM, 128), 128, 0, st>>>(params, w.G, w.m, w.v, ++t, lr);
            count_launch();
        }
    }
    // final loss over the whole set
    k_mlp_fwd<<<n, NH, 0, st>>>(params, X, nullptr, n, w.alpha, nullptr, nullptr, nullptr);
    k_mlp_loss<<<1, 256, 0, st>>>(w.alpha, y, nullptr, n, w.loss);
    count_launch(2);
    float l = 0.f;
    cudaMemcpyAsync(&l, w.loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(dperm, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return mlp_err(THC_CPD_ERR_CUDA, "training failed");
    if (final_loss_host) *final_loss_host = l;
    return THC_CPD_OK;
}
