// FMA throughput probe (include/fr_probe.h).
#include <cuda_runtime.h>

#include "fr_probe.h"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void k_fma_chains(T *out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run(int iters, double *flops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  const int threads = 256, blocks = sms * 8;
  T *buf = nullptr;
  if (cudaMalloc(&buf, sizeof(T) * threads * blocks) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const T a = (T)0.999999, b = (T)1e-7;
  k_fma_chains<T><<<blocks, threads>>>(buf, iters / 10 + 1, a, b);   // warm-up
  cudaEventRecord(e0);
  k_fma_chains<T><<<blocks, threads>>>(buf, iters, a, b);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (err != cudaSuccess || ms <= 0.f) return 1;
  *flops = 2.0 * kChains * (double)iters * threads * blocks / (ms * 1e-3);
  return 0;
}

}  // namespace

extern "C" int32_t fr_probe_fma(int32_t precision, int32_t iters, double *flops) {
  if (!flops || iters < 1) return 1;
  if (precision == 0) return run<double>(iters, flops);
  if (precision == 1) return run<float>(iters, flops);
  return 1;
}
