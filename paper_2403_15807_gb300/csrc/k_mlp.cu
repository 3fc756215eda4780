// k_mlp.cu -- the plan-selection network: 6 -> 64 -> 64 -> 3, ReLU, linear
// output (one predicted log-latency per scan plan), trained with a masked
// mean squared error and Adam.  The paper leaves access-path selection to
// "an optimizer (or a user)" driven by selectivity, dimension and batch
// (Sec. 5.2 / 5.3 takeaways); this network is that optimizer's cost model.
//
// Parameters (float32), row-major: W1[64x6] b1[64] W2[64x64] b2[64]
// W3[3x64] b3[3] (4803 values).
//
// Kernels:
//   mlp_forward   one thread per sample; weights in shared memory; float32,
//                 or bf16 inference (weights, inputs and activations rounded
//                 to bf16, float32 accumulation);
//   mlp_delta     one thread per sample: forward, output error, and the
//                 back-propagated deltas of both hidden layers, stored per
//                 sample together with the activations;
//   mlp_param_grad one thread per parameter: sums its gradient over the
//                 samples (deterministic, no atomics); one extra thread sums
//                 the loss;
//   mlp_adam      one thread per parameter (Kingma & Ba, Algorithm 1).
// The C-ABI entry points (vrs_mlp_*) take host arrays: the data sets are
// small (thousands of samples) and uploaded once per call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/vrs.h"
#include "vrs_internal.cuh"

namespace vrs {
vrs_status set_error(vrs_status st, const char *msg);
}

using namespace vrs;

namespace {

constexpr int IN = 6, H1 = 64, H2 = 64, OUT = 3;
constexpr int NP = H1 * IN + H1 + H2 * H1 + H2 + OUT * H2 + OUT;   // 4803
constexpr int OW1 = 0, OB1 = OW1 + H1 * IN, OW2 = OB1 + H1, OB2 = OW2 + H2 * H1,
              OW3 = OB2 + H2, OB3 = OW3 + OUT * H2;

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

template <bool BF>
__device__ __forceinline__ float rnd(float x) {
    if constexpr (BF) return bf(x);
    return x;
}

// Forward of one sample; a1/a2 (if given) receive the activations.
template <bool BF>
__device__ __forceinline__ void forward1(const float *P, const float *x, float *a1, float *a2,
                                         float *y) {
    float h1[H1];
#pragma unroll 8
    for (int r = 0; r < H1; ++r) {
        float s = P[OB1 + r];
#pragma unroll
        for (int c = 0; c < IN; ++c) s = fmaf(rnd<BF>(P[OW1 + r * IN + c]), rnd<BF>(x[c]), s);
        h1[r] = rnd<BF>(fmaxf(s, 0.0f));
        if (a1) a1[r] = h1[r];
    }
    float yo[OUT];
#pragma unroll
    for (int o = 0; o < OUT; ++o) yo[o] = P[OB3 + o];
    for (int r = 0; r < H2; ++r) {
        float s = P[OB2 + r];
#pragma unroll 16
        for (int c = 0; c < H1; ++c) s = fmaf(rnd<BF>(P[OW2 + r * H1 + c]), h1[c], s);
        const float h = rnd<BF>(fmaxf(s, 0.0f));
        if (a2) a2[r] = h;
#pragma unroll
        for (int o = 0; o < OUT; ++o) yo[o] = fmaf(rnd<BF>(P[OW3 + o * H2 + r]), h, yo[o]);
    }
#pragma unroll
    for (int o = 0; o < OUT; ++o) y[o] = yo[o];
}

__device__ inline void load_params(float *Ps, const float *P) {
    for (int i = threadIdx.x; i < NP; i += blockDim.x) Ps[i] = P[i];
    __syncthreads();
}

template <bool BF>
__global__ void mlp_forward_kernel(const float *__restrict__ P, const float *__restrict__ X,
                                   int64_t m, float *__restrict__ Y) {
    __shared__ float Ps[NP];
    load_params(Ps, P);
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    forward1<BF>(Ps, X + j * IN, nullptr, nullptr, Y + j * OUT);
}

// Per sample: activations a1, a2, output deltas d3 = 2 w (y - t) / msum, and
// hidden deltas d2 = (W3^T d3) . [a2 > 0], d1 = (W2^T d2) . [a1 > 0];
// loss_j = sum_o w (y - t)^2 / msum.
__global__ void mlp_delta_kernel(const float *__restrict__ P, const float *__restrict__ X,
                                 const float *__restrict__ T, const float *__restrict__ M,
                                 int64_t m, float inv_msum, float *__restrict__ A1,
                                 float *__restrict__ A2, float *__restrict__ D1,
                                 float *__restrict__ D2, float *__restrict__ D3,
                                 float *__restrict__ L) {
    __shared__ float Ps[NP];
    load_params(Ps, P);
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    float *a1 = A1 + j * H1, *a2 = A2 + j * H2;
    float y[OUT];
    forward1<false>(Ps, X + j * IN, a1, a2, y);
    float d3[OUT], loss = 0.0f;
#pragma unroll
    for (int o = 0; o < OUT; ++o) {
        const float w = M[j * OUT + o], e = y[o] - T[j * OUT + o];
        loss += w * e * e * inv_msum;
        d3[o] = 2.0f * w * e * inv_msum;
        D3[j * OUT + o] = d3[o];
    }
    L[j] = loss;
    float d2[H2];
    for (int c = 0; c < H2; ++c) {
        float s = 0.0f;
#pragma unroll
        for (int o = 0; o < OUT; ++o) s = fmaf(Ps[OW3 + o * H2 + c], d3[o], s);
        d2[c] = a2[c] > 0.0f ? s : 0.0f;
        D2[j * H2 + c] = d2[c];
    }
    for (int c = 0; c < H1; ++c) {
        float s = 0.0f;
#pragma unroll 16
        for (int r = 0; r < H2; ++r) s = fmaf(Ps[OW2 + r * H1 + c], d2[r], s);
        D1[j * H1 + c] = a1[c] > 0.0f ? s : 0.0f;
    }
}

// One thread per parameter (index < NP) sums its gradient over samples;
// thread NP sums the loss.
__global__ void mlp_param_grad_kernel(const float *__restrict__ X, const float *__restrict__ A1,
                                      const float *__restrict__ A2, const float *__restrict__ D1,
                                      const float *__restrict__ D2, const float *__restrict__ D3,
                                      const float *__restrict__ L, int64_t m,
                                      float *__restrict__ G, float *__restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > NP) return;
    float s = 0.0f;   // accumulation order fixed by the sample index
    if (p == NP) {
        for (int64_t j = 0; j < m; ++j) s += L[j];
        *loss = s;
        return;
    }
    if (p < OB1) {
        const int r = p / IN, c = p % IN;
        for (int64_t j = 0; j < m; ++j) s += D1[j * H1 + r] * X[j * IN + c];
    } else if (p < OW2) {
        const int r = p - OB1;
        for (int64_t j = 0; j < m; ++j) s += D1[j * H1 + r];
    } else if (p < OB2) {
        const int r = (p - OW2) / H1, c = (p - OW2) % H1;
        for (int64_t j = 0; j < m; ++j) s += D2[j * H2 + r] * A1[j * H1 + c];
    } else if (p < OW3) {
        const int r = p - OB2;
        for (int64_t j = 0; j < m; ++j) s += D2[j * H2 + r];
    } else if (p < OB3) {
        const int o = (p - OW3) / H2, c = (p - OW3) % H2;
        for (int64_t j = 0; j < m; ++j) s += D3[j * OUT + o] * A2[j * H2 + c];
    } else {
        const int o = p - OB3;
        for (int64_t j = 0; j < m; ++j) s += D3[j * OUT + o];
    }
    G[p] = s;
}

__global__ void mlp_adam_kernel(float *__restrict__ P, const float *__restrict__ G,
                                float *__restrict__ M1, float *__restrict__ M2, int t, float lr,
                                float b1, float b2, float eps) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const float g = G[p];
    const float m1 = b1 * M1[p] + (1.0f - b1) * g;
    const float m2 = b2 * M2[p] + (1.0f - b2) * g * g;
    M1[p] = m1;
    M2[p] = m2;
    const float mh = m1 / (1.0f - powf(b1, (float)t));
    const float vh = m2 / (1.0f - powf(b2, (float)t));
    P[p] -= lr * mh / (sqrtf(vh) + eps);
}

// Device copies of one data set plus the per-sample work arrays.
struct MlpWork {
    float *P = nullptr, *X = nullptr, *T = nullptr, *M = nullptr, *A1 = nullptr, *A2 = nullptr,
          *D1 = nullptr, *D2 = nullptr, *D3 = nullptr, *L = nullptr, *G = nullptr, *M1 = nullptr,
          *M2 = nullptr, *loss = nullptr;
    ~MlpWork() {
        float *all[] = {P, X, T, M, A1, A2, D1, D2, D3, L, G, M1, M2, loss};
        for (float *p : all)
            if (p) cudaFree(p);
    }
};

#define ML_CK(call)                                                                    \
    do {                                                                               \
        if ((call) != cudaSuccess) {                                                   \
            cudaGetLastError();                                                        \
            return set_error(VRS_ECUDA, "vrs_mlp: " #call " failed");                  \
        }                                                                              \
    } while (0)

vrs_status setup(MlpWork &w, const float *params, const float *X, const float *T,
                 const float *M, int64_t m, bool grad) {
    auto alloc = [&](float **p, size_t n) { return cudaMalloc(p, std::max<size_t>(n, 1) * 4); };
    ML_CK(alloc(&w.P, NP));
    ML_CK(alloc(&w.X, (size_t)m * IN));
    ML_CK(cudaMemcpy(w.P, params, NP * 4, cudaMemcpyHostToDevice));
    ML_CK(cudaMemcpy(w.X, X, (size_t)m * IN * 4, cudaMemcpyHostToDevice));
    if (!grad) return VRS_OK;
    ML_CK(alloc(&w.T, (size_t)m * OUT));
    ML_CK(alloc(&w.M, (size_t)m * OUT));
    ML_CK(alloc(&w.A1, (size_t)m * H1));
    ML_CK(alloc(&w.A2, (size_t)m * H2));
    ML_CK(alloc(&w.D1, (size_t)m * H1));
    ML_CK(alloc(&w.D2, (size_t)m * H2));
    ML_CK(alloc(&w.D3, (size_t)m * OUT));
    ML_CK(alloc(&w.L, (size_t)m));
    ML_CK(alloc(&w.G, NP));
    ML_CK(alloc(&w.M1, NP));
    ML_CK(alloc(&w.M2, NP));
    ML_CK(alloc(&w.loss, 1));
    ML_CK(cudaMemcpy(w.T, T, (size_t)m * OUT * 4, cudaMemcpyHostToDevice));
    ML_CK(cudaMemcpy(w.M, M, (size_t)m * OUT * 4, cudaMemcpyHostToDevice));
    ML_CK(cudaMemset(w.M1, 0, NP * 4));
    ML_CK(cudaMemset(w.M2, 0, NP * 4));
    return VRS_OK;
}

vrs_status grad_step(MlpWork &w, int64_t m, float inv_msum) {
    const int tb = 128;
    mlp_delta_kernel<<<(unsigned)((m + tb - 1) / tb), tb>>>(w.P, w.X, w.T, w.M, m, inv_msum, w.A1,
                                                            w.A2, w.D1, w.D2, w.D3, w.L);
    ML_CK(cudaGetLastError());
    mlp_param_grad_kernel<<<(NP + 1 + 255) / 256, 256>>>(w.X, w.A1, w.A2, w.D1, w.D2, w.D3, w.L,
                                                         m, w.G, w.loss);
    ML_CK(cudaGetLastError());
    return VRS_OK;
}

float mask_sum(const float *M, int64_t m) {
    double s = 0.0;
    for (int64_t i = 0; i < m * OUT; ++i) s += M[i];
    return (float)s;
}

}  // namespace

extern "C" {

VRS_API int32_t vrs_mlp_nparams(void) { return NP; }

VRS_API vrs_status vrs_mlp_forward(const float *params, const float *X, int64_t m, int32_t bf16,
                                   float *Y) {
    if (!params || !X || !Y || m < 1) return set_error(VRS_EINVAL, "vrs_mlp_forward: bad argument");
    MlpWork w;
    vrs_status st = setup(w, params, X, nullptr, nullptr, m, false);
    if (st != VRS_OK) return st;
    float *Yd = nullptr;
    ML_CK(cudaMalloc(&Yd, (size_t)m * OUT * 4));
    const int tb = 128;
    if (bf16)
        mlp_forward_kernel<true><<<(unsigned)((m + tb - 1) / tb), tb>>>(w.P, w.X, m, Yd);
    else
        mlp_forward_kernel<false><<<(unsigned)((m + tb - 1) / tb), tb>>>(w.P, w.X, m, Yd);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(Y, Yd, (size_t)m * OUT * 4, cudaMemcpyDeviceToHost);
    cudaFree(Yd);
    if (e != cudaSuccess) return set_error(VRS_ECUDA, "vrs_mlp_forward: kernel failed");
    return VRS_OK;
}

VRS_API vrs_status vrs_mlp_grad(const float *params, const float *X, const float *T,
                                const float *M, int64_t m, float *grad, float *loss) {
    if (!params || !X || !T || !M || !grad || !loss || m < 1)
        return set_error(VRS_EINVAL, "vrs_mlp_grad: bad argument");
    const float ms = mask_sum(M, m);
    if (!(ms > 0.0f)) return set_error(VRS_EINVAL, "vrs_mlp_grad: the mask is all zero");
    MlpWork w;
    vrs_status st = setup(w, params, X, T, M, m, true);
    if (st != VRS_OK) return st;
    st = grad_step(w, m, 1.0f / ms);
    if (st != VRS_OK) return st;
    ML_CK(cudaMemcpy(grad, w.G, NP * 4, cudaMemcpyDeviceToHost));
    ML_CK(cudaMemcpy(loss, w.loss, 4, cudaMemcpyDeviceToHost));
    return VRS_OK;
}

VRS_API vrs_status vrs_mlp_train(float *params, const float *X, const float *T, const float *M,
                                 int64_t m, int32_t steps, float lr, float *loss_out) {
    if (!params || !X || !T || !M || m < 1 || steps < 0 || !(lr > 0.0f))
        return set_error(VRS_EINVAL, "vrs_mlp_train: bad argument");
    const float ms = mask_sum(M, m);
    if (!(ms > 0.0f)) return set_error(VRS_EINVAL, "vrs_mlp_train: the mask is all zero");
    MlpWork w;
    vrs_status st = setup(w, params, X, T, M, m, true);
    if (st != VRS_OK) return st;
    for (int t = 1; t <= steps; ++t) {
        st = grad_step(w, m, 1.0f / ms);
        if (st != VRS_OK) return st;
        mlp_adam_kernel<<<(NP + 255) / 256, 256>>>(w.P, w.G, w.M1, w.M2, t, lr, 0.9f, 0.999f,
                                                  1e-8f);
        ML_CK(cudaGetLastError());
    }
    // loss at the final parameters
    st = grad_step(w, m, 1.0f / ms);
    if (st != VRS_OK) return st;
    ML_CK(cudaMemcpy(params, w.P, NP * 4, cudaMemcpyDeviceToHost));
    if (loss_out) ML_CK(cudaMemcpy(loss_out, w.loss, 4, cudaMemcpyDeviceToHost));
    return VRS_OK;
}

}  // extern "C"
