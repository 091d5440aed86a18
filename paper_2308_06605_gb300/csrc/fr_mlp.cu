// Training kernels of the eddy-viscosity network (include/fr.h, fr_mlp_*), FP32.
//
// Network (see fr_set_closure): x^ = (x - mean)/std, three GELU layers of 64, z = w4.h3 + b4,
// prediction softplus(z).  Loss = mean over the n samples of (softplus(z) - y)^2.  Backpropagation
// is written out layer by layer: deltas da_l = (W_{l+1}^T da_{l+1}) * gelu'(a_l), weight gradients
// sum da_l (x) h_{l-1} over the samples.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "fr.h"

namespace {

constexpr int NIN = 11, NH = 64;
// Offsets in the flat parameter vector.
constexpr int oW1 = 0, ob1 = oW1 + NH * NIN, oW2 = ob1 + NH, ob2 = oW2 + NH * NH, oW3 = ob2 + NH, ob3 = oW3 + NH * NH,
              ow4 = ob3 + NH, ob4 = ow4 + NH, NPAR = ob4 + 1;
static_assert(NPAR == FR_CLOSURE_NPARAMS, "parameter layout");
// Workspace per sample: a1 h1 a2 h2 a3 h3 (64 each), z, dz.
constexpr int WS = 6 * NH + 2;

__device__ __forceinline__ float gelu(float a) { return 0.5f * a * (1.f + erff(a * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_prime(float a) {
  return 0.5f * (1.f + erff(a * 0.70710678118654752f)) + a * 0.39894228040143268f * expf(-0.5f * a * a);
}
__device__ __forceinline__ float softplus(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }
__device__ __forceinline__ float sigmoid(float z) { return 1.f / (1.f + expf(-z)); }

// Hidden layer l (1..3): a = W in + b, h = gelu(a), thread per (sample, neuron).
__global__ void k_fwd_hidden(const float *__restrict__ P, const float *__restrict__ X, const float *__restrict__ sc,
                             float *__restrict__ work, int64_t n, int layer) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * NH) return;
  const int64_t s = t / NH;
  const int j = (int)(t % NH);
  float *ws = work + s * WS;
  float a;
  if (layer == 1) {
    a = P[ob1 + j];
    for (int k = 0; k < NIN; ++k) a = fmaf(P[oW1 + j * NIN + k], (X[s * NIN + k] - sc[k]) / sc[NIN + k], a);
  } else {
    const int oW = layer == 2 ? oW2 : oW3, ob = layer == 2 ? ob2 : ob3;
    const float *hin = ws + (layer == 2 ? 1 : 3) * NH;
    a = P[ob + j];
    for (int k = 0; k < NH; ++k) a = fmaf(P[oW + j * NH + k], hin[k], a);
  }
  float *aout = ws + (2 * (layer - 1)) * NH;
  aout[j] = a;
  aout[NH + j] = gelu(a);
}

// Output: z, prediction (forward only) or loss and dz (training).
__global__ void k_fwd_out(const float *__restrict__ P, float *__restrict__ work, int64_t n,
                          const float *__restrict__ y, float *__restrict__ pred, float *__restrict__ loss) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float *ws = work + s * WS;
  const float *h3 = ws + 5 * NH;
  float z = P[ob4];
  for (int k = 0; k < NH; ++k) z = fmaf(P[ow4 + k], h3[k], z);
  ws[6 * NH] = z;
  const float sp = softplus(z);
  if (pred) pred[s] = sp;
  if (y) {
    const float r = sp - y[s];
    ws[6 * NH + 1] = 2.f * r * sigmoid(z) / (float)n;
    atomicAdd(loss, r * r / (float)n);
  }
}

// Delta of hidden layer l from the layer above (in place over a_l): thread per (sample, neuron).
__global__ void k_back_delta(const float *__restrict__ P, float *__restrict__ work, int64_t n, int layer) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * NH) return;
  const int64_t s = t / NH;
  const int k = (int)(t % NH);
  float *ws = work + s * WS;
  float g;
  if (layer == 3) {
    g = ws[6 * NH + 1] * P[ow4 + k];
  } else {
    const int oW = layer == 2 ? oW3 : oW2;
    const float *dnext = ws + (2 * layer) * NH;    // delta of layer + 1, stored over its a
    g = 0.f;
    for (int j = 0; j < NH; ++j) g = fmaf(P[oW + j * NH + k], dnext[j], g);
  }
  float *a = ws + (2 * (layer - 1)) * NH;
  a[k] = g * gelu_prime(a[k]);
}

// Weight and bias gradients of one layer: thread per (neuron j, input k), summing over samples.
__global__ void k_weight_grad(const float *__restrict__ work, const float *__restrict__ X, const float *__restrict__ sc,
                              float *__restrict__ grad, int64_t n, int layer) {
  const int K = layer == 1 ? NIN : NH;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (layer == 4) {
    if (t > NH) return;
    float g = 0.f;
    for (int64_t s = 0; s < n; ++s) {
      const float *ws = work + s * WS;
      g += ws[6 * NH + 1] * (t < NH ? ws[5 * NH + t] : 1.f);
    }
    grad[t < NH ? ow4 + t : ob4] = g;
    return;
  }
  if (t >= NH * (K + 1)) return;
  const int j = t / (K + 1), k = t % (K + 1);   // k == K: bias
  const int oW = layer == 1 ? oW1 : (layer == 2 ? oW2 : oW3), ob = layer == 1 ? ob1 : (layer == 2 ? ob2 : ob3);
  float g = 0.f;
  for (int64_t s = 0; s < n; ++s) {
    const float *ws = work + s * WS;
    const float d = ws[(2 * (layer - 1)) * NH + j];
    float in;
    if (k == K) in = 1.f;
    else if (layer == 1) in = (X[s * NIN + k] - sc[k]) / sc[NIN + k];
    else in = ws[(2 * (layer - 2) + 1) * NH + k];
    g = fmaf(d, in, g);
  }
  grad[k == K ? ob + j : oW + j * K + k] = g;
}

__global__ void k_adam(float *__restrict__ P, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float mi = b1 * m[i] + (1.f - b1) * g[i];
  const float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

fr_status forward_pass(const float *P, const float *X, const float *sc, int64_t n, float *work, cudaStream_t st) {
  const unsigned gb = (unsigned)((n * NH + 255) / 256);
  for (int layer = 1; layer <= 3; ++layer) k_fwd_hidden<<<gb, 256, 0, st>>>(P, X, sc, work, n, layer);
  return cudaGetLastError() == cudaSuccess ? FR_OK : FR_ECUDA;
}

}  // namespace

extern "C" int64_t fr_mlp_workspace_floats(int64_t n) { return n * WS + 1; }

extern "C" fr_status fr_mlp_forward(const float *params, const float *scales, const float *X, int64_t n, float *out,
                                    float *work, uintptr_t stream) {
  if (!params || !scales || !X || !out || !work || n < 1) return FR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (forward_pass(params, X, scales, n, work, st) != FR_OK) return FR_ECUDA;
  k_fwd_out<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(params, work, n, nullptr, out, nullptr);
  return cudaGetLastError() == cudaSuccess ? FR_OK : FR_ECUDA;
}

extern "C" fr_status fr_mlp_loss_grad(const float *params, const float *scales, const float *X, const float *y,
                                      int64_t n, float *grad, float *loss, float *work, uintptr_t stream) {
  if (!params || !scales || !X || !y || !grad || !loss || !work || n < 1) return FR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess) return FR_ECUDA;
  if (forward_pass(params, X, scales, n, work, st) != FR_OK) return FR_ECUDA;
  k_fwd_out<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(params, work, n, y, nullptr, loss);
  const unsigned gb = (unsigned)((n * NH + 255) / 256);
  k_weight_grad<<<1, 128, 0, st>>>(work, X, scales, grad, n, 4);
  for (int layer = 3; layer >= 1; --layer) {
    k_back_delta<<<gb, 256, 0, st>>>(params, work, n, layer);
    const int K = layer == 1 ? NIN : NH;
    k_weight_grad<<<(NH * (K + 1) + 127) / 128, 128, 0, st>>>(work, X, scales, grad, n, layer);
  }
  return cudaGetLastError() == cudaSuccess ? FR_OK : FR_ECUDA;
}

extern "C" fr_status fr_mlp_adam(float *params, const float *grad, float *m, float *v, int32_t n_params, float lr,
                                 float beta1, float beta2, float eps, int32_t step, uintptr_t stream) {
  if (!params || !grad || !m || !v || n_params < 1 || step < 1) return FR_EINVAL;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adam<<<(n_params + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, n_params, lr, beta1, beta2, eps,
                                                                    c1, c2);
  return cudaGetLastError() == cudaSuccess ? FR_OK : FR_ECUDA;
}
