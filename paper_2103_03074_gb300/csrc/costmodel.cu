// Learned cost model: a small MLP that predicts log2 of a contraction step's
// device time from the step's features, trained on the step-timing recorder's
// measurements by this file's own forward, backward and Adam kernels.
//
// Network: x (kFeat = 16) -> 64 ReLU -> 64 ReLU -> 1, FP32.  Parameters are
// one flat array: W1[64][16], b1[64], W2[64][64], b2[64], w3[64], b3.
// Loss: mean squared error of the prediction against log2(ms).
//
// fwdbwd_kernel: one CTA per 64 samples keeps the weights, the activations
// and their gradients in shared memory, computes each weight gradient as a
// sum over the CTA's samples (one thread per gradient element) and adds it
// into the global gradient with one atomic per element and CTA.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "costmodel.h"
#include "kernels.h"
#include "tn_internal.h"

namespace tn {

namespace {

constexpr int F = kCostFeatures, H1 = 64, H2 = 64;
constexpr int oW1 = 0, oB1 = oW1 + H1 * F, oW2 = oB1 + H1, oB2 = oW2 + H2 * H1, oW3 = oB2 + H2, oB3 = oW3 + H2;
constexpr int kParams = oB3 + 1;
constexpr int S = 64;     // samples per CTA
constexpr int LD = 65;    // padded row stride of the activation tiles
constexpr int kThreads = 256;
constexpr size_t kSmem = sizeof(float) * (kParams + S * F + 4 * S * LD + S);

struct Tiles {
    float *w, *x, *h1, *h2, *d2, *d1, *dy;
};

__device__ Tiles carve(float *smem) {
    Tiles t;
    t.w = smem;
    t.x = t.w + kParams;
    t.h1 = t.x + S * F;
    t.h2 = t.h1 + S * LD;
    t.d2 = t.h2 + S * LD;
    t.d1 = t.d2 + S * LD;
    t.dy = t.d1 + S * LD;
    return t;
}

// forward pass of the CTA's samples into the shared tiles; returns nothing,
// leaves y in dy[] (before the loss gradient overwrites it)
__device__ void forward_tiles(const Tiles &t, const float *__restrict__ params, const float *__restrict__ X,
                              int64_t s0, int nv) {
    for (int i = threadIdx.x; i < kParams; i += blockDim.x) t.w[i] = params[i];
    for (int i = threadIdx.x; i < S * F; i += blockDim.x) {
        const int s = i / F;
        t.x[i] = s < nv ? X[(s0 + s) * F + (i % F)] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < S * H1; i += blockDim.x) {
        const int s = i / H1, j = i % H1;
        float a = t.w[oB1 + j];
        for (int k = 0; k < F; k++) a = fmaf(t.w[oW1 + j * F + k], t.x[s * F + k], a);
        t.h1[s * LD + j] = fmaxf(a, 0.f);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < S * H2; i += blockDim.x) {
        const int s = i / H2, j = i % H2;
        float a = t.w[oB2 + j];
        for (int k = 0; k < H1; k++) a = fmaf(t.w[oW2 + j * H1 + k], t.h1[s * LD + k], a);
        t.h2[s * LD + j] = fmaxf(a, 0.f);
    }
    __syncthreads();
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        float a = t.w[oB3];
        for (int k = 0; k < H2; k++) a = fmaf(t.w[oW3 + k], t.h2[s * LD + k], a);
        t.dy[s] = a;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads) predict_kernel(const float *params, const float *X, float *Y, int64_t n) {
    extern __shared__ float smem[];
    const Tiles t = carve(smem);
    const int64_t s0 = (int64_t)blockIdx.x * S;
    const int nv = (int)(n - s0 < S ? n - s0 : S);
    forward_tiles(t, params, X, s0, nv);
    for (int s = threadIdx.x; s < nv; s += blockDim.x) Y[s0 + s] = t.dy[s];
}

__global__ void __launch_bounds__(kThreads) fwdbwd_kernel(const float *params, const float *X, const float *T,
                                                          int64_t n, float *grad, double *loss) {
    extern __shared__ float smem[];
    const Tiles t = carve(smem);
    const int64_t s0 = (int64_t)blockIdx.x * S;
    const int nv = (int)(n - s0 < S ? n - s0 : S);
    forward_tiles(t, params, X, s0, nv);
    const float scale = 2.0f / (float)n;
    // dL/dy = 2 (y - t) / n for valid samples
    if (threadIdx.x < 32) {
        double l = 0.0;
        for (int s = threadIdx.x; s < S; s += 32) {
            float d = 0.f;
            if (s < nv) {
                d = t.dy[s] - T[s0 + s];
                l += (double)d * d;
            }
            t.dy[s] = d * scale;
        }
        for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
        if (threadIdx.x == 0) atomicAdd(loss, l / (double)n);
    }
    __syncthreads();
    // dh2 = dy w3 (ReLU mask)
    for (int i = threadIdx.x; i < S * H2; i += blockDim.x) {
        const int s = i / H2, j = i % H2;
        t.d2[s * LD + j] = t.h2[s * LD + j] > 0.f ? t.dy[s] * t.w[oW3 + j] : 0.f;
    }
    __syncthreads();
    // dh1 = W2^T dh2 (ReLU mask); gradients of layer 3 and layer 2
    for (int i = threadIdx.x; i < S * H1; i += blockDim.x) {
        const int s = i / H1, k = i % H1;
        float a = 0.f;
        if (t.h1[s * LD + k] > 0.f)
            for (int j = 0; j < H2; j++) a = fmaf(t.w[oW2 + j * H1 + k], t.d2[s * LD + j], a);
        t.d1[s * LD + k] = a;
    }
    for (int j = threadIdx.x; j < H2; j += blockDim.x) {
        float g = 0.f;
        for (int s = 0; s < S; s++) g = fmaf(t.dy[s], t.h2[s * LD + j], g);
        atomicAdd(&grad[oW3 + j], g);
    }
    if (threadIdx.x == 0) {
        float g = 0.f;
        for (int s = 0; s < S; s++) g += t.dy[s];
        atomicAdd(&grad[oB3], g);
    }
    for (int i = threadIdx.x; i < H2 * H1; i += blockDim.x) {
        const int j = i / H1, k = i % H1;
        float g = 0.f;
        for (int s = 0; s < S; s++) g = fmaf(t.d2[s * LD + j], t.h1[s * LD + k], g);
        atomicAdd(&grad[oW2 + i], g);
    }
    for (int j = threadIdx.x; j < H2; j += blockDim.x) {
        float g = 0.f;
        for (int s = 0; s < S; s++) g += t.d2[s * LD + j];
        atomicAdd(&grad[oB2 + j], g);
    }
    __syncthreads();
    // gradients of layer 1
    for (int i = threadIdx.x; i < H1 * F; i += blockDim.x) {
        const int j = i / F, k = i % F;
        float g = 0.f;
        for (int s = 0; s < S; s++) g = fmaf(t.d1[s * LD + j], t.x[s * F + k], g);
        atomicAdd(&grad[oW1 + i], g);
    }
    for (int j = threadIdx.x; j < H1; j += blockDim.x) {
        float g = 0.f;
        for (int s = 0; s < S; s++) g += t.d1[s * LD + j];
        atomicAdd(&grad[oB1 + j], g);
    }
}

// Adam (Kingma & Ba 2015) with bias correction
__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

int cost_params() { return kParams; }

}  // namespace tn

struct tn_costmodel {
    float *d_params = nullptr, *d_grad = nullptr, *d_m = nullptr, *d_v = nullptr;
    double *d_loss = nullptr;
    int64_t steps = 0;
};

namespace tn {
namespace {

int cuda_err(cudaError_t e, const char *what) {
    return fail(TN_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

cudaError_t set_attrs() {
    cudaError_t e = set_max_dynamic_smem((const void *)fwdbwd_kernel, (int)kSmem);
    if (e == cudaSuccess) e = set_max_dynamic_smem((const void *)predict_kernel, (int)kSmem);
    return e;
}

}  // namespace

// host helper used by the order search: predictions for a host feature matrix
int cost_predict_host(tn_costmodel_t cm, const std::vector<float> &X, std::vector<float> &Y) {
    const int64_t n = (int64_t)(X.size() / F);
    Y.assign(n, 0.f);
    if (n == 0) return TN_OK;
    float *dX = nullptr, *dY = nullptr;
    cudaError_t e = cudaMalloc(&dX, X.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dY, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(dX, X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = set_attrs();
    if (e == cudaSuccess) {
        predict_kernel<<<(unsigned)((n + S - 1) / S), kThreads, kSmem>>>(cm->d_params, dX, dY, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(Y.data(), dY, n * sizeof(float), cudaMemcpyDeviceToHost);
    if (dX) cudaFree(dX);
    if (dY) cudaFree(dY);
    return e == cudaSuccess ? TN_OK : cuda_err(e, "cost model prediction");
}

}  // namespace tn

using namespace tn;

extern "C" int tn_costmodel_create(tn_costmodel_t *out, uint64_t seed) {
    if (!out) return fail(TN_ERR_ARG, "out is NULL");
    *out = nullptr;
    // He-normal weights from SplitMix64 + Box-Muller, zero biases
    std::vector<float> p(kParams, 0.f);
    uint64_t st = seed;
    auto next = [&]() {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto normal = [&]() {
        const double u1 = 1.0 - (double)(next() >> 11) * (1.0 / 9007199254740992.0);
        const double u2 = (double)(next() >> 11) * (1.0 / 9007199254740992.0);
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    for (int i = 0; i < H1 * F; i++) p[oW1 + i] = (float)(normal() * std::sqrt(2.0 / F));
    for (int i = 0; i < H2 * H1; i++) p[oW2 + i] = (float)(normal() * std::sqrt(2.0 / H1));
    for (int i = 0; i < H2; i++) p[oW3 + i] = (float)(normal() * std::sqrt(1.0 / H2));
    tn_costmodel *cm = new tn_costmodel();
    cudaError_t e = cudaMalloc(&cm->d_params, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&cm->d_grad, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&cm->d_m, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&cm->d_v, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&cm->d_loss, sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(cm->d_params, p.data(), kParams * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(cm->d_m, 0, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(cm->d_v, 0, kParams * sizeof(float));
    if (e != cudaSuccess) {
        tn_costmodel_destroy(cm);
        return cuda_err(e, "tn_costmodel_create");
    }
    *out = cm;
    return TN_OK;
}

extern "C" void tn_costmodel_destroy(tn_costmodel_t cm) {
    if (!cm) return;
    cudaFree(cm->d_params);
    cudaFree(cm->d_grad);
    cudaFree(cm->d_m);
    cudaFree(cm->d_v);
    cudaFree(cm->d_loss);
    delete cm;
}

extern "C" int tn_costmodel_params(tn_costmodel_t cm, float *get, const float *set, int *n_params) {
    if (!cm) return fail(TN_ERR_ARG, "cost model is NULL");
    if (n_params) *n_params = kParams;
    cudaError_t e = cudaSuccess;
    if (set) e = cudaMemcpy(cm->d_params, set, kParams * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && get) e = cudaMemcpy(get, cm->d_params, kParams * sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? TN_OK : cuda_err(e, "tn_costmodel_params");
}

extern "C" int tn_costmodel_grad(tn_costmodel_t cm, const float *d_X, const float *d_T, int64_t n, float *d_grad,
                                 double *loss, tn_stream_t stream) {
    if (!cm || !d_X || !d_T || n <= 0) return fail(TN_ERR_ARG, "tn_costmodel_grad: bad arguments");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = set_attrs();
    if (e == cudaSuccess) e = cudaMemsetAsync(cm->d_grad, 0, kParams * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cm->d_loss, 0, sizeof(double), s);
    if (e == cudaSuccess) {
        fwdbwd_kernel<<<(unsigned)((n + S - 1) / S), kThreads, kSmem, s>>>(cm->d_params, d_X, d_T, n, cm->d_grad,
                                                                           cm->d_loss);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && d_grad)
        e = cudaMemcpyAsync(d_grad, cm->d_grad, kParams * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && loss) {
        e = cudaMemcpyAsync(loss, cm->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    return e == cudaSuccess ? TN_OK : cuda_err(e, "tn_costmodel_grad");
}

extern "C" int tn_costmodel_train(tn_costmodel_t cm, const float *d_X, const float *d_T, int64_t n, int epochs,
                                  float lr, double *final_loss, tn_stream_t stream) {
    if (!cm || !d_X || !d_T || n <= 0 || epochs < 0) return fail(TN_ERR_ARG, "tn_costmodel_train: bad arguments");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = set_attrs();
    const float b1 = 0.9f, b2 = 0.999f;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ep++) {
        e = cudaMemsetAsync(cm->d_grad, 0, kParams * sizeof(float), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(cm->d_loss, 0, sizeof(double), s);
        if (e != cudaSuccess) break;
        fwdbwd_kernel<<<(unsigned)((n + S - 1) / S), kThreads, kSmem, s>>>(cm->d_params, d_X, d_T, n, cm->d_grad,
                                                                           cm->d_loss);
        cm->steps++;
        const float c1 = 1.f - std::pow(b1, (float)cm->steps), c2 = 1.f - std::pow(b2, (float)cm->steps);
        adam_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(cm->d_params, cm->d_grad, cm->d_m, cm->d_v, kParams, lr,
                                                          b1, b2, 1e-8f, c1, c2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && final_loss) {
        e = cudaMemcpyAsync(final_loss, cm->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    return e == cudaSuccess ? TN_OK : cuda_err(e, "tn_costmodel_train");
}

extern "C" int tn_costmodel_predict(tn_costmodel_t cm, const float *d_X, float *d_Y, int64_t n, tn_stream_t stream) {
    if (!cm || !d_X || !d_Y || n < 0) return fail(TN_ERR_ARG, "tn_costmodel_predict: bad arguments");
    if (n == 0) return TN_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = set_attrs();
    if (e == cudaSuccess) {
        predict_kernel<<<(unsigned)((n + S - 1) / S), kThreads, kSmem, s>>>(cm->d_params, d_X, d_Y, n);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? TN_OK : cuda_err(e, "tn_costmodel_predict");
}
