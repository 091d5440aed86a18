// Device bodies of the hexahedral FR kernels, shared by the per-mesh kernels (fr_kernels.cu)
// and the batched persistent stage kernel (fr_batch_kernel.cu).  Everything here has internal
// linkage: each translation unit that includes it holds its own copy, including the constant-
// memory basis tables, which each unit uploads through its upload_basis_local().
//
// Kernels of the FR residual and the RK44 stage update (arXiv 2308.06605, section "FR
// Algorithm", Eq. 1-3).  One residual evaluation is four launches (plus two for boundary faces):
//   interp_faces : Q -> solution traces at the flux points of every face (interface slots)
//   bc_prepare   : boundary faces: common solution Q^I and ghost traces
//   volume       : per element, BR2-corrected gradients, physical + transformed fluxes at the
//                  solution points, gradient traces at the flux points, and the divergence of
//                  the transformed flux including the own-flux part of the correction
//   iface_flux   : per interface flux point, Rusanov + BR2 common normal flux (bc_flux for
//                  boundary faces)
//   correct      : per solution point, adds the common-flux correction, scales by -1/|J| and
//                  writes R or applies the RK44 stage update (always FP64).
//
// Every kernel is a template on the scalar type T of its element arithmetic and of the arrays it
// exchanges: T = double is the FP64 path; T = df32 (FP32 hi + lo pairs on the FP32 pipe) is the
// mixed path, in which the Riemann flux's pressure/energy recovery, the boundary states and the
// RK update stay FP64.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include <cuda_bf16.h>

#include "df32.cuh"
#include "fr_device.hpp"
#include "fr_point.cuh"
#include "fr_prism_bodies.cuh"

namespace frx {
namespace {

template <typename T>
struct BasisT {
  T D[kMaxN * kMaxN];    // D[i*N + a] = l_a'(x_i)
  T Dt[kMaxN * kMaxN];   // D - hp (x) lp + hm (x) lm: divergence with the own-flux correction
  T lm[kMaxN], lp[kMaxN], hm[kMaxN], hp[kMaxN];
  double w[kMaxN];       // Gauss-Legendre weights (closure's element means)
};

__constant__ BasisT<double> c_basis_d[kMaxN];   // index N - 1
__constant__ BasisT<df32> c_basis_f[kMaxN];

template <typename T> __device__ __forceinline__ const BasisT<T> &cbasis(int N);
template <> __device__ __forceinline__ const BasisT<double> &cbasis<double>(int N) { return c_basis_d[N - 1]; }
template <> __device__ __forceinline__ const BasisT<df32> &cbasis<df32>(int N) { return c_basis_f[N - 1]; }

// 1D tables of one order in both element arithmetics.
inline void fill_basis(const Basis1D &b, BasisT<double> &d, BasisT<df32> &f) {
  const int N = b.N;
  d = BasisT<double>{};
  f = BasisT<df32>{};
  for (int i = 0; i < N; ++i) {
    d.lm[i] = b.lm[i];
    d.lp[i] = b.lp[i];
    d.hm[i] = b.hm[i];
    d.hp[i] = b.hp[i];
    d.w[i] = b.w[i];
    for (int a = 0; a < N; ++a) {
      d.D[i * N + a] = b.D[i * N + a];
      d.Dt[i * N + a] = b.D[i * N + a] - b.hp[i] * b.lp[a] + b.hm[i] * b.lm[a];
    }
  }
  for (int i = 0; i < kMaxN; ++i) {
    f.lm[i] = df_split_host(d.lm[i]);
    f.lp[i] = df_split_host(d.lp[i]);
    f.hm[i] = df_split_host(d.hm[i]);
    f.hp[i] = df_split_host(d.hp[i]);
    f.w[i] = d.w[i];
  }
  for (int i = 0; i < kMaxN * kMaxN; ++i) {
    f.D[i] = df_split_host(d.D[i]);
    f.Dt[i] = df_split_host(d.Dt[i]);
  }
}

// Upload of this translation unit's copy of the 1D basis tables (constant memory is per unit);
// DG-equivalent correction.
cudaError_t upload_basis_local() {
  BasisT<double> hd[kMaxN] = {};
  BasisT<df32> hf[kMaxN] = {};
  for (int p = 1; p < kMaxN; ++p) fill_basis(make_basis(p), hd[p], hf[p]);
  cudaError_t e = cudaMemcpyToSymbol(c_basis_d, hd, sizeof(hd));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_basis_f, hf, sizeof(hf));
}

// Tables of the kernels: the constant-memory DG-equivalent ones, or (VC) the mesh's own copy in
// global memory for a correction function c != 0 of the energy-stable family.
template <int N, typename T, bool VC>
__device__ __forceinline__ const BasisT<T> &basis_ref(const DevPhys &dph) {
  if constexpr (VC)
    return *reinterpret_cast<const BasisT<T> *>(dph.vc_basis);
  else
    return cbasis<T>(N);
}

// Strides of the reference axes in the point index m = i + N j + N^2 k.
template <int N>
__device__ __forceinline__ int axis_stride(int a) {
  return a == 0 ? 1 : (a == 1 ? N : N * N);
}

// Flux point r = a + N b of face f: base index of its normal line and the stride along it.
template <int N>
__device__ __forceinline__ void face_line(int f, int r, int &base, int &sd) {
  const int d = f >> 1;
  const int t0 = (d == 0) ? 1 : 0, t1 = (d == 2) ? 1 : 2;
  const int a = r % N, b = r / N;
  base = a * axis_stride<N>(t0) + b * axis_stride<N>(t1);
  sd = axis_stride<N>(d);
}

__device__ __forceinline__ int slot_of(int code, int a, int b, int N) {
  if (code & 4) { int t = a; a = b; b = t; }
  if (code & 1) a = N - 1 - a;
  if (code & 2) b = N - 1 - b;
  return a + N * b;
}

// Eddy-viscosity network for one element, evaluated by one warp (lane = 0..31): BF16 weights,
// FP32 activations and accumulation.  x: the 11 raw features; buf: 128 floats of shared memory.
// Returns nu_t = s_out Delta^2 softplus(z) (Delta = x[10]).
__device__ __forceinline__ float closure_mlp(const DevPhys &dph, const float x_raw[11], float *buf, int lane) {
  const __nv_bfloat16 *W = static_cast<const __nv_bfloat16 *>(dph.cw);
  const float *sc = dph.cscale;
  float x[11];
#pragma unroll
  for (int c = 0; c < 11; ++c) x[c] = (x_raw[c] - sc[c]) / sc[11 + c];
  const __nv_bfloat16 *W1 = W, *b1 = W1 + 64 * 11, *W2 = b1 + 64, *b2 = W2 + 64 * 64, *W3 = b2 + 64,
                      *b3 = W3 + 64 * 64, *w4 = b3 + 64, *b4 = w4 + 64;
  float *hA = buf, *hB = buf + 64;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int n = lane + 32 * r;
    float a = __bfloat162float(b1[n]);
#pragma unroll
    for (int c = 0; c < 11; ++c) a = fmaf(__bfloat162float(W1[n * 11 + c]), x[c], a);
    hA[n] = 0.5f * a * (1.f + erff(a * 0.70710678118654752f));
  }
  __syncwarp();
  const __nv_bfloat16 *Ws[2] = {W2, W3}, *bs[2] = {b2, b3};
  float *hin = hA, *hout = hB;
#pragma unroll
  for (int layer = 0; layer < 2; ++layer) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int n = lane + 32 * r;
      float a = __bfloat162float(bs[layer][n]);
      for (int c = 0; c < 64; ++c) a = fmaf(__bfloat162float(Ws[layer][n * 64 + c]), hin[c], a);
      hout[n] = 0.5f * a * (1.f + erff(a * 0.70710678118654752f));
    }
    __syncwarp();
    float *t = hin;
    hin = hout;
    hout = t;
  }
  float z = __bfloat162float(w4[lane]) * hin[lane] + __bfloat162float(w4[lane + 32]) * hin[lane + 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
  z += __bfloat162float(b4[0]);
  const float sp = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));
  __syncwarp();
  return sc[22] * x_raw[10] * x_raw[10] * sp;
}

// ------------------------------------------------------------------------------------------
// 1. Solution traces.  Thread per (element, face, flux point).
// ------------------------------------------------------------------------------------------
template <int N, typename T>
__device__ __forceinline__ void interp_body(int64_t t, const T *__restrict__ Q, const int32_t *__restrict__ ef,
                                            T *__restrict__ Qtr, int64_t E) {
  constexpr int Np = N * N * N, Nf = N * N;
  if (t >= E * 6 * Nf) return;
  const int r = (int)(t % Nf);
  const int64_t eff = t / Nf;
  const int f = (int)(eff % 6);
  const int64_t e = eff / 6;
  const BasisT<T> &B = cbasis<T>(N);
  const T *l = (f & 1) ? B.lp : B.lm;
  int base, sd;
  face_line<N>(f, r, base, sd);
  const T *q = Q + e * Np * 5;
  Dot<T> acc[5];
#pragma unroll
  for (int c = 0; c < N; ++c) {
    const T lc = l[c];
    const T *qc = q + (base + c * sd) * 5;
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v].add(lc, qc[v]);
  }
  const int packed = ef[eff];
  const int64_t I = packed >> 4;
  const int side = (packed >> 3) & 1;
  const int slot = slot_of(packed & 7, r % N, r / N, N);
  T *dst = Qtr + (I * 2 + side) * 5 * Nf + slot;
#pragma unroll
  for (int v = 0; v < 5; ++v) dst[v * Nf] = acc[v].get();
}

template <int N, typename T>
__global__ void k_interp_faces(const T *__restrict__ Q, const int32_t *__restrict__ ef,
                               T *__restrict__ Qtr, int64_t E) {
  interp_body<N, T>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, Q, ef, Qtr, E);
}

// The same interpolation with the elements' states staged through shared memory: a block of
// kInterpThreads threads loads interp_epb<N>() consecutive elements with coalesced reads (the
// point-major [pt][v] layout of consecutive elements is one contiguous range), then computes
// their face traces from shared memory.
constexpr int kInterpThreads = 256;
template <int N>
__host__ __device__ constexpr int interp_epb() {
  return (2 * kInterpThreads) / (6 * N * N) < 1 ? 1
         : ((2 * kInterpThreads) / (6 * N * N) > 16 ? 16 : (2 * kInterpThreads) / (6 * N * N));
}

template <int N, typename T>
__global__ void __launch_bounds__(kInterpThreads)
    k_interp_faces_smem(const T *__restrict__ Q, const int32_t *__restrict__ ef, T *__restrict__ Qtr, int64_t E) {
  constexpr int Np = N * N * N, Nf = N * N, EPB = interp_epb<N>();
  __shared__ T sq[EPB * 5 * Np];     // [element][v][point]
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int ne = (int)(E - e0 < EPB ? E - e0 : EPB);
  const T *src = Q + e0 * Np * 5;
  for (int idx = threadIdx.x; idx < ne * Np * 5; idx += kInterpThreads) {
    const int le = idx / (Np * 5), rem = idx - le * Np * 5;
    sq[(le * 5 + rem % 5) * Np + rem / 5] = src[idx];
  }
  __syncthreads();
  const BasisT<T> &B = cbasis<T>(N);
  for (int t = threadIdx.x; t < ne * 6 * Nf; t += kInterpThreads) {
    const int le = t / (6 * Nf), fr_ = t - le * 6 * Nf;
    const int f = fr_ / Nf, r = fr_ % Nf;
    const T *l = (f & 1) ? B.lp : B.lm;
    int base, sd;
    face_line<N>(f, r, base, sd);
    const T *q = sq + le * 5 * Np + base;
    Dot<T> acc[5];
#pragma unroll
    for (int c = 0; c < N; ++c) {
      const T lc = l[c];
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v].add(lc, q[v * Np + c * sd]);
    }
    const int packed = ef[(e0 + le) * 6 + f];
    const int64_t I = packed >> 4;
    const int side = (packed >> 3) & 1;
    const int slot = slot_of(packed & 7, r % N, r / N, N);
    T *dst = Qtr + (I * 2 + side) * 5 * Nf + slot;
#pragma unroll
    for (int v = 0; v < 5; ++v) dst[v * Nf] = acc[v].get();
  }
}

// ------------------------------------------------------------------------------------------
// 2. Volume kernel.  One block per element, one thread per solution point.
// ------------------------------------------------------------------------------------------
template <int N>
constexpr int volume_threads() { return ((N * N * N + 31) / 32) * 32; }
// Resident blocks the register budget must allow (smem allows at least this many).
template <int N>
constexpr int volume_min_blocks() {
  // Measured on GB300: 16 warps per SM (128 registers) is fastest for the 32- and 64-thread
  // blocks of p = 2, 3 and, with the per-variable gradient and the contravariant fluxes, for the
  // 128-thread blocks of p = 4 (4 blocks, no spills in double-float; 3 blocks of 168 registers
  // were 3 % slower); p = 1 keeps 8 blocks (16 would spill).
  return N == 2 ? 8 : (N == 5 ? 4 : (volume_threads<N>() <= 128 ? 512 / volume_threads<N>()
                                                                 : (volume_threads<N>() <= 256 ? 2 : 1)));
}

// Shared-memory values (of T) one element needs in the volume kernel.
template <int N>
__host__ __device__ constexpr int volume_smem_values() { return 35 * N * N * N + 30 * N * N; }

// One element e handled by `nth` threads of the block (thread index tid in [0, nth)); every
// thread of the block calls this together (it contains block barriers); inactive sub-blocks
// (active = false) only take part in the barriers.
template <int N, typename T, bool VC = false, bool FP32V = false>
__device__ __forceinline__ void volume_body(int64_t e, int tid, int nth, bool active, double *sm_raw,
                                            const T *__restrict__ Q, const T *__restrict__ metrics,
                                            const int32_t *__restrict__ ef, const T *__restrict__ Qtr,
                                            const T *__restrict__ liftfac, T *__restrict__ Gtr,
                                            T *__restrict__ Rpart, const DevPhys &dph,
                                            const double *__restrict__ hel, float *__restrict__ nu_out,
                                            const int8_t *__restrict__ if_up, int64_t n_interior) {
  constexpr int Np = N * N * N, Nf = N * N;
  using TG = typename GradOf<T, FP32V>::type;   // arithmetic of the viscous branch
  constexpr bool kPert = !std::is_same<TG, T>::value;
  T *sm = reinterpret_cast<T *>(sm_raw);
  T *sQ = sm;                                                // [5][Np]
  TG *sG = reinterpret_cast<TG *>(sQ + 5 * Np);              // [15][Np] uncorrected physical gradient, j*5+v
  T *sH = sQ + 20 * Np;                                      // [15][Np] transformed flux, index d*5+v
  TG *sdQ = reinterpret_cast<TG *>(sH + 15 * Np);            // [6][5][Nf] Q^I - Q_own at the flux points
  // FP32 viscous branch: Q minus the element's first point, in FP32, in the upper half of the
  // gradient buffer (the FP32 gradient uses only its lower half).
  TG *sQg = kPert ? reinterpret_cast<TG *>(sQ + 5 * Np) + 15 * Np : nullptr;   // [5][Np]
  const PhysT<T> &ph = phys_of<T>(dph);
  const PhysT<TG> &phg = phys_of<TG>(dph);
  const BasisT<T> &B = basis_ref<N, T, VC>(dph);
  // Sums of products end with Dot::raw(): the compensated sum s + e renormalised by one
  // fast_two_sum only (an error of the order of 2^-48 of the sum of the terms' magnitudes).
  const bool viscous = dph.viscous != 0;
  const bool pt = active && tid < Np;
  const int m = tid < Np ? tid : 0, i = m % N, j = (m / N) % N, k = m / (N * N);
  // The point's metric terms are loaded before the staging loops so that their latency overlaps them.
  T S[9], invJ, q[5];
  if (pt) {
    const T *met = metrics + e * 10 * Np + m;
#pragma unroll
    for (int c = 0; c < 9; ++c) S[c] = met[c * Np];
    invJ = met[9 * Np];
  }
  if (active)
    for (int t = tid; t < 5 * Np; t += nth) {
      const T x = Q[e * Np * 5 + t];
      sQ[(t % 5) * Np + t / 5] = x;
      if constexpr (kPert)
        if (viscous) sQg[(t % 5) * Np + t / 5] = to_g<TG>(x - Q[e * Np * 5 + t % 5]);
    }
  if (viscous && active) {
    for (int t = tid; t < 6 * Nf; t += nth) {
      const int f = t / Nf, r = t % Nf;
      const int packed = ef[e * 6 + f];
      const int64_t I = packed >> 4;
      const int side = (packed >> 3) & 1;
      const int slot = slot_of(packed & 7, r % N, r / N, N);
      const T *own = Qtr + (I * 2 + side) * 5 * Nf + slot;
      const T *oth = Qtr + (I * 2 + (1 - side)) * 5 * Nf + slot;
      // Q^I - Q_own.  BR2: (other - own)/2 (a boundary's other slot holds 2 Q^I - Q-).  LDG: 0 on
      // the side that supplies Q^I, other - own on the other; boundaries as BR2.
      T w = ph.half;
      if (dph.ldg && I < n_interior) w = side == (if_up[I] ? 0 : 1) ? ph.zero : ph.one;
#pragma unroll
      for (int v = 0; v < 5; ++v) sdQ[(f * 5 + v) * Nf + r] = to_g<TG>(w * (oth[v * Nf] - own[v * Nf]));
    }
  }
  __syncthreads();
  TG G[15];
  if (pt) {
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v] = sQ[v * Np + m];
    if (viscous) {
      // One variable at a time: reference gradient, its correction, and both transformed to
      // physical components at once (short live ranges; the same operations as a two-pass form).
      TG sj[9];   // S[d][jj] / |J|
#pragma unroll
      for (int c = 0; c < 9; ++c) sj[c] = to_g<TG>(S[c] * invJ);
      const TG nhm[3] = {-to_g<TG>(B.hm[i]), -to_g<TG>(B.hm[j]), -to_g<TG>(B.hm[k])};
      // The variable loop stays rolled (a smaller instruction footprint): the corrected gradient
      // goes through shared memory, in this thread's own entries of the transformed-flux buffer,
      // which only this thread writes later (R gradient values of type TG per entry of type T).
      constexpr int R = sizeof(T) / sizeof(TG);
      TG *sGc = reinterpret_cast<TG *>(sH);
      auto gslot = [&](int c) { return ((c / R) * Np + m) * R + c % R; };
#pragma unroll 1
      for (int v = 0; v < 5; ++v) {
        const TG *sq;
        if constexpr (kPert)
          sq = sQg + v * Np;
        else
          sq = sQ + v * Np;
        Dot<TG> a0, a1, a2;
#pragma unroll
        for (int a = 0; a < N; ++a) {
          a0.add(to_g<TG>(B.D[i * N + a]), sq[a + N * j + N * N * k]);
          a1.add(to_g<TG>(B.D[j * N + a]), sq[i + N * a + N * N * k]);
          a2.add(to_g<TG>(B.D[k * N + a]), sq[i + N * j + N * N * a]);
        }
        const TG gu0 = a0.raw(), gu1 = a1.raw(), gu2 = a2.raw();
        a0.add(nhm[0], sdQ[(0 * 5 + v) * Nf + j + N * k]);
        a0.add(to_g<TG>(B.hp[i]), sdQ[(1 * 5 + v) * Nf + j + N * k]);
        a1.add(nhm[1], sdQ[(2 * 5 + v) * Nf + i + N * k]);
        a1.add(to_g<TG>(B.hp[j]), sdQ[(3 * 5 + v) * Nf + i + N * k]);
        a2.add(nhm[2], sdQ[(4 * 5 + v) * Nf + i + N * j]);
        a2.add(to_g<TG>(B.hp[k]), sdQ[(5 * 5 + v) * Nf + i + N * j]);
        const TG gc0 = a0.raw(), gc1 = a1.raw(), gc2 = a2.raw();
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
          Dot<TG> du, dc;
          du.add(sj[0 * 3 + jj], gu0);
          du.add(sj[1 * 3 + jj], gu1);
          du.add(sj[2 * 3 + jj], gu2);
          dc.add(sj[0 * 3 + jj], gc0);
          dc.add(sj[1 * 3 + jj], gc1);
          dc.add(sj[2 * 3 + jj], gc2);
          const TG gc = dc.raw();
          sGc[gslot(jj * 5 + v)] = gc;
          // Face-gradient source: BR2 the uncorrected gradient (+ eta r_f), LDG the corrected one.
          sG[(jj * 5 + v) * Np + m] = dph.ldg ? gc : du.raw();
        }
      }
#pragma unroll
      for (int c = 0; c < 15; ++c) G[c] = sGc[gslot(c)];
    }
  }
  T rho_nu = ph.zero;
  if (viscous && dph.closure) {
    // Eddy-viscosity closure: quadrature-weighted element mean of the corrected velocity
    // gradient, then one warp evaluates the network (BF16 weights, FP32 accumulation).
    float *red = reinterpret_cast<float *>(sm + volume_smem_values<N>());   // [10][Np] + 129
    if (pt) {
      const double ri = 1.0 / to_double(q[0]);
      const double w = (double)B.w[i] * B.w[j] * B.w[k] / to_double(invJ);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const double dudx = (to_double(G[b * 5 + 1 + a]) - to_double(q[1 + a]) * ri * to_double(G[b * 5])) * ri;
          red[(a * 3 + b) * Np + m] = (float)(w * dudx);
        }
      red[9 * Np + m] = (float)w;
    }
    __syncthreads();
    if (active && tid < 32) {
      float acc[10];
#pragma unroll
      for (int c = 0; c < 10; ++c) {
        float sacc = 0.f;
        for (int mm = tid; mm < Np; mm += 32) sacc += red[c * Np + mm];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
        acc[c] = sacc;
      }
      float x[11];
      float ss = 0.f;
#pragma unroll
      for (int c = 0; c < 9; ++c) x[c] = acc[c] / acc[9];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const float sab = 0.5f * (x[a * 3 + b] + x[b * 3 + a]);
          ss += sab * sab;
        }
      x[9] = sqrtf(2.f * ss);
      x[10] = (float)(hel[e] / N);
      const float nu = closure_mlp(dph, x, red + 10 * Np + 1, tid);
      if (tid == 0) {
        red[10 * Np] = nu;
        if (nu_out) nu_out[e] = nu;
      }
    }
    __syncthreads();
    if (pt) rho_nu = q[0] * from_double<T>((double)red[10 * Np]);
  }
  if (pt) {
    // Transformed fluxes per reference direction from the contravariant velocity.
    const T ri = ph.one / q[0];
    const T u[3] = {q[1] * ri, q[2] * ri, q[3] * ri};
    const T p = ph.gm1 * (q[4] - ph.half * (q[1] * u[0] + q[2] * u[1] + q[3] * u[2]));
    T tau[3][3], hq[3];
    if (viscous) {
      if constexpr (kPert) {
        TG qg[5], ug[3], taug[3][3], hqg[3];
#pragma unroll
        for (int v = 0; v < 5; ++v) qg[v] = to_g<TG>(q[v]);
        const TG rig = phg.one / qg[0];
#pragma unroll
        for (int c = 0; c < 3; ++c) ug[c] = qg[1 + c] * rig;
        viscous_stress<TG>(qg, ug, rig, G, phg, visc_with(phg, to_g<TG>(rho_nu), dph), taug, hqg);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          hq[a] = from_g<T>(hqg[a]);
#pragma unroll
          for (int b2 = 0; b2 < 3; ++b2) tau[a][b2] = from_g<T>(taug[a][b2]);
        }
      } else {
        viscous_stress<T>(q, u, ri, G, ph, visc_with(ph, rho_nu, dph), tau, hq);
      }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      T f[5];
      contravariant_flux<T>(q, u, p, S + 3 * d, viscous, tau, hq, f);
#pragma unroll
      for (int v = 0; v < 5; ++v) sH[(d * 5 + v) * Np + m] = f[v];
    }
  }
  __syncthreads();
  if (viscous && active) {
    // Gradient traces: uncorrected gradient interpolated to the face + eta * own lifting.
    // One item per (gradient component jj, face point): 3 * 6 * Nf items keep the block busy.
    for (int t = tid; t < 18 * Nf; t += nth) {
      const int jj = t / (6 * Nf), fr_ = t - jj * 6 * Nf;
      const int f = fr_ / Nf, r = fr_ % Nf;
      const T *l = (f & 1) ? B.lp : B.lm;
      int base, sd;
      face_line<N>(f, r, base, sd);
      const int packed = ef[e * 6 + f];
      const int64_t I = packed >> 4;
      const int side = (packed >> 3) & 1;
      const int slot = slot_of(packed & 7, r % N, r / N, N);
      T *dst = Gtr + (I * 2 + side) * 15 * Nf + slot;
      const TG lj = to_g<TG>(ph.eta * liftfac[((e * 6 + f) * 3 + jj) * Nf + r]);
      TG lg[N];
#pragma unroll
      for (int c = 0; c < N; ++c) lg[c] = to_g<TG>(l[c]);
#pragma unroll 1
      for (int v = 0; v < 5; ++v) {
        const TG *sg = sG + (jj * 5 + v) * Np + base;
        Dot<TG> acc;
#pragma unroll
        for (int c = 0; c < N; ++c) acc.add(lg[c], sg[c * sd]);
        acc.add(lj, sdQ[(f * 5 + v) * Nf + r]);
        dst[(jj * 5 + v) * Nf] = from_g<T>(acc.raw());
      }
    }
  }
  if (active && tid < Np) {
    const int m = tid, i = m % N, j = (m / N) % N, k = m / (N * N);
    T *out = Rpart + (e * Np + m) * 5;
#pragma unroll 1
    for (int v = 0; v < 5; ++v) {
      const T *h0 = sH + (0 * 5 + v) * Np, *h1 = sH + (1 * 5 + v) * Np, *h2 = sH + (2 * 5 + v) * Np;
      Dot<T> acc;
#pragma unroll
      for (int a = 0; a < N; ++a) {
        acc.add(B.Dt[i * N + a], h0[a + N * j + N * N * k]);
        acc.add(B.Dt[j * N + a], h1[i + N * a + N * N * k]);
        acc.add(B.Dt[k * N + a], h2[i + N * j + N * N * a]);
      }
      out[v] = acc.raw();
    }
  }
}

// Resident blocks at p = 5 and 6: 3 blocks of 224 and (double-float) 2 of 352 threads at 80
// registers, with some spills, measured faster than the register-limited 2 and 1 (double-float
// p = 6: 9.16 -> 7.73 ms per launch at 40^3; p = 5: 8.80 -> 8.61 ms at 48^3; FP64 p = 5: 25.63 ->
// 25.26 ms; FP64 p = 6 unchanged at 2 blocks, so it keeps 1).
template <int N, typename T>
constexpr int volume_min_blocks_of() {
  return N == 6 ? 3 : ((N == 7 && !std::is_same<T, double>::value) ? 2 : volume_min_blocks<N>());
}

// With the viscous branch in FP32 (96 registers, no spills) the kernels of p = 3 and 4 fit 10 and
// 5 blocks per SM, which hides more of their load latency (p = 4: 6.44 -> 5.96 ms per launch at
// 64^3; p = 3: 3.27 -> 3.00 ms); the double-float ones measured slower at those counts.
template <int N, typename T, bool FP32V>
constexpr int volume_min_blocks_v() {
  return (FP32V && N == 5) ? 5 : ((FP32V && N == 4) ? 10 : volume_min_blocks_of<N, T>());
}

template <int N, typename T, bool FP32V = false>
__global__ void __launch_bounds__(volume_threads<N>(), volume_min_blocks_v<N, T, FP32V>())
    k_volume(const T *__restrict__ Q, const T *__restrict__ metrics, const int32_t *__restrict__ ef,
             const T *__restrict__ Qtr, const T *__restrict__ liftfac, T *__restrict__ Gtr, T *__restrict__ Rpart,
             DevPhys dph, const double *__restrict__ hel, float *__restrict__ nu_out,
             const int8_t *__restrict__ if_up, int64_t n_interior) {
  extern __shared__ double sm_raw[];
  volume_body<N, T, false, FP32V>(blockIdx.x, threadIdx.x, blockDim.x, true, sm_raw, Q, metrics, ef, Qtr, liftfac, Gtr,
                                  Rpart, dph, hel, nu_out, if_up, n_interior);
}

// ------------------------------------------------------------------------------------------
// 3. Common normal flux at the flux points of two-sided interfaces (Rusanov + BR2).  The
// inviscid part (pressure/energy recovery) is FP64 in both paths.
// ------------------------------------------------------------------------------------------
template <int N, typename T, bool FP32V = false>
__device__ __forceinline__ void iface_body(int64_t t, const T *__restrict__ Qtr, const T *__restrict__ Gtr,
                                           const T *__restrict__ normals, T *__restrict__ FI, int64_t n_if,
                                           const DevPhys &dph, const int32_t *__restrict__ if_elem,
                                           const float *__restrict__ nu, const int8_t *__restrict__ if_up) {
  constexpr int Nf = N * N;
  if (t >= n_if * Nf) return;
  const int64_t I = t / Nf;
  const int q = (int)(t % Nf);
  const PhysT<T> &ph = phys_of<T>(dph);
  T qL[5], qR[5], nT[3];
  const T nn = normals[(I * 4 + 3) * Nf + q];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qL[v] = Qtr[(I * 2 + 0) * 5 * Nf + v * Nf + q];
    qR[v] = Qtr[(I * 2 + 1) * 5 * Nf + v * Nf + q];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) nT[c] = normals[(I * 4 + c) * Nf + q];
  T F[5];
  if (dph.inviscid == FR_ROE) {
    double a[5], b[5], nd[3], Fd[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      a[v] = to_double(qL[v]);
      b[v] = to_double(qR[v]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) nd[c] = to_double(nT[c]);
    roe_flux(a, b, nd, to_double(nn), dph.gamma, Fd);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = from_double<T>(Fd[v]);
  } else {
    T fL[5], fR[5], sL, sR;
    normal_inviscid(qL, nT, nn, dph, fL, sL);
    normal_inviscid(qR, nT, nn, dph, fR, sR);
    const T hl = ph.half * fmax(sL, sR);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = ph.half * (fL[v] + fR[v]) - hl * (qR[v] - qL[v]);
  }
  if constexpr (!std::is_same<typename GradOf<T, FP32V>::type, T>::value) {
    if (dph.viscous) {
      // FR_PREC_MIXED_VF32: the whole viscous part in FP32 (the gradient traces written by the
      // volume kernel's FP32 branch are exact FP32 values).
      using TG = typename GradOf<T, FP32V>::type;
      const PhysT<TG> &phg = phys_of<TG>(dph);
      TG qg[5], Gg[15], ng[3], Fv[3][5];
      const int sup = (dph.ldg && if_up[I]) ? 0 : 1;
#pragma unroll
      for (int v = 0; v < 5; ++v)
        qg[v] = dph.ldg ? to_g<TG>(sup == 0 ? qL[v] : qR[v]) : phg.half * (to_g<TG>(qL[v]) + to_g<TG>(qR[v]));
#pragma unroll
      for (int c = 0; c < 15; ++c) {
        const TG g0 = to_g<TG>(Gtr[(I * 2 + 0) * 15 * Nf + c * Nf + q]);
        const TG g1 = to_g<TG>(Gtr[(I * 2 + 1) * 15 * Nf + c * Nf + q]);
        Gg[c] = dph.ldg ? (sup == 0 ? g1 : g0) : phg.half * (g0 + g1);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) ng[c] = to_g<TG>(nT[c]);
      TG rho_nu = phg.zero;
      if (dph.closure) rho_nu = qg[0] * (TG)(0.5 * ((double)nu[if_elem[2 * I]] + (double)nu[if_elem[2 * I + 1]]));
      viscous_flux<TG>(qg, Gg, phg, visc_with(phg, rho_nu, dph), Fv);
#pragma unroll
      for (int v = 0; v < 5; ++v) F[v] -= from_g<T>(Fv[0][v] * ng[0] + Fv[1][v] * ng[1] + Fv[2][v] * ng[2]);
      if (dph.ldg) {
        const T tn = ph.tau * nn;
#pragma unroll
        for (int v = 0; v < 5; ++v) F[v] += tn * (qL[v] - qR[v]);
      }
    }
  } else if (dph.viscous) {
    T qc[5], G[15];
    if (dph.ldg) {
      // LDG: the supplying side's solution, the other side's gradient.
      const int sup = if_up[I] ? 0 : 1;
#pragma unroll
      for (int v = 0; v < 5; ++v) qc[v] = sup == 0 ? qL[v] : qR[v];
#pragma unroll
      for (int c = 0; c < 15; ++c) G[c] = Gtr[(I * 2 + (1 - sup)) * 15 * Nf + c * Nf + q];
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) qc[v] = ph.half * (qL[v] + qR[v]);
#pragma unroll
      for (int c = 0; c < 15; ++c)
        G[c] = ph.half * (Gtr[(I * 2 + 0) * 15 * Nf + c * Nf + q] + Gtr[(I * 2 + 1) * 15 * Nf + c * Nf + q]);
    }
    T rho_nu = ph.zero;
    if (dph.closure) rho_nu = qc[0] * from_double<T>(0.5 * ((double)nu[if_elem[2 * I]] + (double)nu[if_elem[2 * I + 1]]));
    T Fv[3][5];
    viscous_flux<T>(qc, G, ph, visc_with(ph, rho_nu, dph), Fv);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] -= Fv[0][v] * nT[0] + Fv[1][v] * nT[1] + Fv[2][v] * nT[2];
    if (dph.ldg) {
      const T tn = ph.tau * nn;
#pragma unroll
      for (int v = 0; v < 5; ++v) F[v] += tn * (qL[v] - qR[v]);
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) FI[(I * 5 + v) * Nf + q] = F[v];
}

// 5 resident blocks of 128 threads (96 registers, a few spills): the double-float interface
// kernel measured 4 % faster than with 128 registers and 4 blocks; the FP64 one is unchanged.
template <int N, typename T, bool FP32V = false>
__global__ void __launch_bounds__(128, 5) k_iface_flux(const T *__restrict__ Qtr, const T *__restrict__ Gtr,
                             const T *__restrict__ normals, T *__restrict__ FI, int64_t n_if, DevPhys dph,
                             const int32_t *__restrict__ if_elem, const float *__restrict__ nu,
                             const int8_t *__restrict__ if_up) {
  iface_body<N, T, FP32V>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, Qtr, Gtr, normals, FI, n_if, dph, if_elem,
                          nu, if_up);
}

// ------------------------------------------------------------------------------------------
// 3b. Boundary faces.  Side 0 of a boundary interface is the element; its side-1 slot holds
// 2 Q^I - Q- so that the volume kernel's (other - own)/2 equals Q^I - Q- for the BR2 jump.
// Boundary states are FP64 in both paths.
// ------------------------------------------------------------------------------------------
// Ghost state (for the Rusanov flux) and boundary common solution Q^I from the interior trace.
__device__ void boundary_states(const double qm[5], const double n[3], double nn, const fr_bc &bc,
                                const DevPhys &ph, double ghost[5], double qi[5]) {
  const double g = ph.gamma, Rg = ph.R;
  const double ri = 1.0 / qm[0];
  const double u[3] = {qm[1] * ri, qm[2] * ri, qm[3] * ri};
  const double p = (g - 1.0) * (qm[4] - 0.5 * (qm[1] * u[0] + qm[2] * u[1] + qm[3] * u[2]));
  if (bc.kind == FR_BC_DIRICHLET) {
    for (int v = 0; v < 5; ++v) ghost[v] = qi[v] = bc.params[v];
    return;
  }
  if (bc.kind == FR_BC_WALL_ISOTHERMAL) {
    ghost[0] = qm[0]; ghost[1] = -qm[1]; ghost[2] = -qm[2]; ghost[3] = -qm[3]; ghost[4] = qm[4];
    qi[0] = qm[0]; qi[1] = qi[2] = qi[3] = 0.0;
    qi[4] = qm[0] * Rg * bc.params[0] / (g - 1.0);
    return;
  }
  const double nh[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
  const double un = u[0] * nh[0] + u[1] * nh[1] + u[2] * nh[2];
  const double c = sqrt(g * p * ri);
  const double Rp = un + 2.0 * c / (g - 1.0);          // outgoing Riemann invariant
  double rb, ub[3], pb;
  if (bc.kind == FR_BC_CHAR_OUTFLOW) {
    pb = bc.params[0];
    const double sent = p / pow(qm[0], g);
    rb = pow(pb / sent, 1.0 / g);
    const double unb = Rp - 2.0 * sqrt(g * pb / rb) / (g - 1.0);
    for (int c3 = 0; c3 < 3; ++c3) ub[c3] = u[c3] + (unb - un) * nh[c3];
  } else {  // FR_BC_CHAR_INFLOW: total pressure, total temperature, direction
    const double p0 = bc.params[0], T0 = bc.params[1];
    double d[3] = {bc.params[2], bc.params[3], bc.params[4]};
    const double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int c3 = 0; c3 < 3; ++c3) d[c3] /= dn;
    const double a = nh[0] * d[0] + nh[1] * d[1] + nh[2] * d[2];
    const double k = 2.0 / (g - 1.0);
    const double A = a * a + k, B = -2.0 * a * Rp, C = Rp * Rp - k * k * g * Rg * T0;
    const double V = (-B + sqrt(B * B - 4.0 * A * C)) / (2.0 * A);
    const double cp = g * Rg / (g - 1.0);
    const double Tb = T0 - V * V / (2.0 * cp);
    pb = p0 * pow(Tb / T0, g / (g - 1.0));
    rb = pb / (Rg * Tb);
    for (int c3 = 0; c3 < 3; ++c3) ub[c3] = V * d[c3];
  }
  qi[0] = rb;
  qi[1] = rb * ub[0];
  qi[2] = rb * ub[1];
  qi[3] = rb * ub[2];
  qi[4] = pb / (g - 1.0) + 0.5 * rb * (ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
  for (int v = 0; v < 5; ++v) ghost[v] = qi[v];
}

template <int N, typename T>
__device__ __forceinline__ void bc_prepare_body(int64_t t, T *__restrict__ Qtr, const T *__restrict__ normals,
                                                const int32_t *__restrict__ if_bc, const fr_bc *__restrict__ bcs,
                                                int64_t first, int64_t count, const DevPhys &ph) {
  constexpr int Nf = N * N;
  if (t >= count * Nf) return;
  const int64_t I = first + t / Nf;
  const int q = (int)(t % Nf);
  double qm[5], n[3], gh[5], qi[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) qm[v] = to_double(Qtr[(I * 2 + 0) * 5 * Nf + v * Nf + q]);
#pragma unroll
  for (int c = 0; c < 3; ++c) n[c] = to_double(normals[(I * 4 + c) * Nf + q]);
  boundary_states(qm, n, to_double(normals[(I * 4 + 3) * Nf + q]), bcs[if_bc[I]], ph, gh, qi);
#pragma unroll
  for (int v = 0; v < 5; ++v) Qtr[(I * 2 + 1) * 5 * Nf + v * Nf + q] = from_double<T>(2.0 * qi[v] - qm[v]);
}

template <int N, typename T>
__global__ void k_bc_prepare(T *__restrict__ Qtr, const T *__restrict__ normals,
                             const int32_t *__restrict__ if_bc, const fr_bc *__restrict__ bcs,
                             int64_t first, int64_t count, DevPhys ph) {
  bc_prepare_body<N, T>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, Qtr, normals, if_bc, bcs, first, count, ph);
}

template <int N, typename T>
__device__ __forceinline__ void bc_flux_body(int64_t t, const T *__restrict__ Qtr, const T *__restrict__ Gtr,
                                             const T *__restrict__ normals, const int32_t *__restrict__ if_bc,
                                             const fr_bc *__restrict__ bcs, T *__restrict__ FI, int64_t first,
                                             int64_t count, const DevPhys &dph,
                                             const int32_t *__restrict__ if_elem, const float *__restrict__ nu) {
  constexpr int Nf = N * N;
  if (t >= count * Nf) return;
  const int64_t I = first + t / Nf;
  const int q = (int)(t % Nf);
  double qm[5], n[3], gh[5], qi[5];
  T nT[3];
#pragma unroll
  for (int v = 0; v < 5; ++v) qm[v] = to_double(Qtr[(I * 2 + 0) * 5 * Nf + v * Nf + q]);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    nT[c] = normals[(I * 4 + c) * Nf + q];
    n[c] = to_double(nT[c]);
  }
  const double nn = to_double(normals[(I * 4 + 3) * Nf + q]);
  boundary_states(qm, n, nn, bcs[if_bc[I]], dph, gh, qi);
  T F[5];
  if (dph.inviscid == FR_ROE) {
    double Fd[5];
    roe_flux(qm, gh, n, nn, dph.gamma, Fd);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = from_double<T>(Fd[v]);
  } else {
    double fL[5], fR[5], sL, sR;
    normal_inviscid(qm, n, nn, dph.gamma, fL, sL);
    normal_inviscid(gh, n, nn, dph.gamma, fR, sR);
    const double lam = fmax(sL, sR);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = from_double<T>(0.5 * (fL[v] + fR[v]) - 0.5 * lam * (gh[v] - qm[v]));
  }
  if (dph.viscous) {
    const PhysT<T> &ph = phys_of<T>(dph);
    T G[15], qiT[5];
#pragma unroll
    for (int c = 0; c < 15; ++c) G[c] = Gtr[(I * 2 + 0) * 15 * Nf + c * Nf + q];
#pragma unroll
    for (int v = 0; v < 5; ++v) qiT[v] = from_double<T>(qi[v]);
    T rho_nu = ph.zero;
    if (dph.closure) rho_nu = qiT[0] * from_double<T>((double)nu[if_elem[2 * I]]);
    T Fv[3][5];
    viscous_flux<T>(qiT, G, ph, visc_with(ph, rho_nu, dph), Fv);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] -= Fv[0][v] * nT[0] + Fv[1][v] * nT[1] + Fv[2][v] * nT[2];
    if (dph.ldg) {
#pragma unroll
      for (int v = 0; v < 5; ++v) F[v] += from_double<T>(dph.ldg_tau * nn * (qm[v] - qi[v]));
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) FI[(I * 5 + v) * Nf + q] = F[v];
}

template <int N, typename T>
__global__ void k_bc_flux(const T *__restrict__ Qtr, const T *__restrict__ Gtr, const T *__restrict__ normals,
                          const int32_t *__restrict__ if_bc, const fr_bc *__restrict__ bcs, T *__restrict__ FI,
                          int64_t first, int64_t count, DevPhys dph, const int32_t *__restrict__ if_elem,
                          const float *__restrict__ nu) {
  bc_flux_body<N, T>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, Qtr, Gtr, normals, if_bc, bcs, FI, first, count,
                     dph, if_elem, nu);
}

// ------------------------------------------------------------------------------------------
// 4. Correction by the common flux, scaling, and output / RK44 stage update (FP64).
// ------------------------------------------------------------------------------------------
template <int N, typename T, bool VC = false>
__device__ __forceinline__ void correct_body(int64_t t, const T *__restrict__ Rpart, const T *__restrict__ FI,
                                             const int32_t *__restrict__ ef, const T *__restrict__ metrics,
                                             int64_t E, int mode, int stage, double dt, double *__restrict__ Rout,
                                             double *__restrict__ Q, T *__restrict__ Qc, double *__restrict__ Un,
                                             T *__restrict__ Unc, double *__restrict__ acc, int *__restrict__ flag,
                                             const DevPhys &dph) {
  constexpr int Np = N * N * N, Nf = N * N;
  if (t >= E * Np) return;
  const int64_t e = t / Np;
  const int m = (int)(t % Np), i = m % N, j = (m / N) % N, k = m / (N * N);
  const BasisT<T> &B = basis_ref<N, T, VC>(dph);
  const PhysT<T> &ph = phys_of<T>(dph);
  Dot<T> r[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) r[v].add(ph.one, Rpart[t * 5 + v]);
  // Faces: (weight, local flux point (a, b)).
  const int fa[6] = {j, j, i, i, i, i};
  const int fb[6] = {k, k, k, k, j, j};
  const T wts[6] = {B.hm[i], B.hp[i], B.hm[j], B.hp[j], B.hm[k], B.hp[k]};
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int packed = ef[e * 6 + f];
    const int64_t I = packed >> 4;
    const int side = (packed >> 3) & 1;
    const int slot = slot_of(packed & 7, fa[f], fb[f], N);
    const T w = side ? -wts[f] : wts[f];
    const T *src = FI + I * 5 * Nf + slot;
#pragma unroll
    for (int v = 0; v < 5; ++v) r[v].add(w, src[v * Nf]);
  }
  const T s = -metrics[(e * 10 + 9) * Np + m];
  T rv[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) rv[v] = r[v].get();
  finish_point<T>(t, rv, s, mode, stage, dt, Rout, Q, Qc, Un, Unc, acc, flag, dph);
}

// 6 resident blocks (40 registers): the double-float kernel measured 2.62 -> 2.55 ms per launch at
// 64^3, p = 4 (its FP64 RK update and its loads overlap better across more warps); FP64 unchanged.
template <int N, typename T>
__global__ void __launch_bounds__(256, 6) k_correct(const T *__restrict__ Rpart, const T *__restrict__ FI, const int32_t *__restrict__ ef,
                          const T *__restrict__ metrics, int64_t E, int mode, int stage, double dt,
                          double *__restrict__ Rout, double *__restrict__ Q, T *__restrict__ Qc,
                          double *__restrict__ Un, T *__restrict__ Unc, double *__restrict__ acc,
                          int *__restrict__ flag, DevPhys dph) {
  correct_body<N, T>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, Rpart, FI, ef, metrics, E, mode, stage, dt, Rout,
                     Q, Qc, Un, Unc, acc, flag, dph);
}

// Meshes with prisms: a triangular interface uses only the first N(N+1)/2 of its N^2 slots;
// these wrappers skip the others before running the interface bodies.
template <int N>
__device__ __forceinline__ bool unused_tri_slot(int64_t t, int64_t first, int64_t count, const int8_t *if_tri) {
  constexpr int Nf = N * N, Nt = N * (N + 1) / 2;
  if (t >= count * Nf) return false;     // out of range: the body's own bound check returns
  return if_tri[first + t / Nf] && (int)(t % Nf) >= Nt;
}

template <int N, typename T>
__global__ void k_iface_flux_tri(const T *__restrict__ Qtr, const T *__restrict__ Gtr, const T *__restrict__ normals,
                                 T *__restrict__ FI, int64_t n_if, DevPhys dph, const int32_t *__restrict__ if_elem,
                                 const float *__restrict__ nu, const int8_t *__restrict__ if_tri,
                                 const int8_t *__restrict__ if_up) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (unused_tri_slot<N>(t, 0, n_if, if_tri)) return;
  iface_body<N, T>(t, Qtr, Gtr, normals, FI, n_if, dph, if_elem, nu, if_up);
}

template <int N, typename T>
__global__ void k_bc_prepare_tri(T *__restrict__ Qtr, const T *__restrict__ normals, const int32_t *__restrict__ if_bc,
                                 const fr_bc *__restrict__ bcs, int64_t first, int64_t count, DevPhys ph,
                                 const int8_t *__restrict__ if_tri) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (unused_tri_slot<N>(t, first, count, if_tri)) return;
  bc_prepare_body<N, T>(t, Qtr, normals, if_bc, bcs, first, count, ph);
}

template <int N, typename T>
__global__ void k_bc_flux_tri(const T *__restrict__ Qtr, const T *__restrict__ Gtr, const T *__restrict__ normals,
                              const int32_t *__restrict__ if_bc, const fr_bc *__restrict__ bcs, T *__restrict__ FI,
                              int64_t first, int64_t count, DevPhys dph, const int32_t *__restrict__ if_elem,
                              const float *__restrict__ nu, const int8_t *__restrict__ if_tri) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (unused_tri_slot<N>(t, first, count, if_tri)) return;
  bc_flux_body<N, T>(t, Qtr, Gtr, normals, if_bc, bcs, FI, first, count, dph, if_elem, nu);
}

// ------------------------------------------------------------------------------------------
// Batched persistent stage: one cooperative launch runs every phase of one RK stage for all
// cases of a ragged ensemble.  Phases are separated by a grid barrier whose waits are bounded:
// a wait that exceeds the spin limit sets the error word and every block returns.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ bool batch_grid_sync(BatchSync *sy, long long limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = &sy->bar_gen;
    volatile int *err = &sy->err;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(&sy->bar_count, 1u) == gridDim.x - 1) {
      atomicExch(&sy->bar_count, 0u);
      __threadfence();
      atomicAdd(&sy->bar_gen, 1u);
    } else {
      long long it = 0;
      while (*gen == g) {
        if (*err) break;
        if (++it > limit) {
          atomicExch(&sy->err, 1);
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int *)&sy->err == 0;
}

template <typename T, int N>
__device__ __forceinline__ void batch_task(const BatchTask &tk, const BatchCase &c, const BatchLaunch &L,
                                           double *smem) {
  const DevMesh &m = c.m;
  const T *Qin = reinterpret_cast<const T *>(m.mixed ? m.Qc : m.Q);
  T *Qtr = reinterpret_cast<T *>(m.Qtr), *Gtr = reinterpret_cast<T *>(m.Gtr), *FI = reinterpret_cast<T *>(m.FI);
  T *Rpart = reinterpret_cast<T *>(m.Rpart);
  const T *met = reinterpret_cast<const T *>(m.metrics), *lift = reinterpret_cast<const T *>(m.liftfac);
  const T *nrm = reinterpret_cast<const T *>(m.normals);
  const int64_t pts = m.E * m.Np * 5;               // first prism value in per-point arrays
  const T *ptab = reinterpret_cast<const T *>(m.ptab), *pmet = reinterpret_cast<const T *>(m.metrics_p);
  const int64_t idx = tk.begin + threadIdx.x < tk.end ? tk.begin + threadIdx.x : (int64_t)1 << 62;
  switch (tk.kind) {
    case TASK_INTERP:
      interp_body<N, T>(tk.begin + threadIdx.x < tk.end ? tk.begin + threadIdx.x : (int64_t)1 << 62, Qin, m.ef, Qtr,
                        m.E);
      break;
    case TASK_BC_PREPARE:
      if (m.if_tri && unused_tri_slot<N>(idx, m.n_interior, m.n_if - m.n_interior, m.if_tri)) break;
      bc_prepare_body<N, T>(idx, Qtr, nrm, m.if_bc, m.bcs, m.n_interior, m.n_if - m.n_interior, c.ph);
      break;
    case TASK_VOLUME: {
      // Sub-blocks of nth threads, one element each; threads past the last full sub-block idle.
      const int tpe = ((N * N * N + 31) / 32) * 32;
      const int nth = tpe >= (int)blockDim.x ? (int)blockDim.x : tpe;
      const int epb = batch_elems_per_block(N, (int)blockDim.x);
      const int le = (int)threadIdx.x / nth;
      const int tid = (int)threadIdx.x % nth;
      const int64_t e = tk.begin + le;
      const bool active = le < epb && e < tk.end;
      volume_body<N, T>(e, tid, nth, active, smem + (size_t)(le < epb ? le : 0) * volume_smem_values<N>(), Qin, met,
                        m.ef, Qtr, lift, Gtr, Rpart, c.ph, m.h, nullptr, m.if_up, m.n_interior);
      break;
    }
    case TASK_IFACE:
      if (m.if_tri && unused_tri_slot<N>(idx, 0, m.n_interior, m.if_tri)) break;
      iface_body<N, T>(idx, Qtr, Gtr, nrm, FI, m.n_interior, c.ph, m.if_elem, m.nu, m.if_up);
      break;
    case TASK_BC_FLUX:
      if (m.if_tri && unused_tri_slot<N>(idx, m.n_interior, m.n_if - m.n_interior, m.if_tri)) break;
      bc_flux_body<N, T>(idx, Qtr, Gtr, nrm, m.if_bc, m.bcs, FI, m.n_interior, m.n_if - m.n_interior, c.ph, m.if_elem,
                         m.nu);
      break;
    case TASK_PRISM_INTERP:
      prism_interp_body<N, T>(idx, Qin + pts, m.ef_p, ptab, m.tri_slot, Qtr, m.Ep);
      break;
    case TASK_PRISM_VOLUME: {
      const int tpe = ((N * (N + 1) / 2 * N + 31) / 32) * 32;
      const int nth = tpe >= (int)blockDim.x ? (int)blockDim.x : tpe;
      const int epb = batch_prism_elems_per_block(N, (int)blockDim.x);
      const int le = (int)threadIdx.x / nth;
      const int tid = (int)threadIdx.x % nth;
      const int64_t e = tk.begin + le;
      const bool active = le < epb && e < tk.end;
      prism_volume_body<N, T>(e, tid, nth, active, smem + (size_t)(le < epb ? le : 0) * prism_smem_values<N>(),
                              Qin + pts, pmet, m.ef_p, Qtr, ptab, m.tri_slot, Gtr, Rpart + pts, c.ph, m.if_up,
                              m.n_interior);
      break;
    }
    case TASK_PRISM_CORRECT:
      prism_correct_body<N, T>(idx, Rpart + pts, FI, m.ef_p, pmet, ptab, m.tri_slot, m.Ep, m.E * m.Np, MODE_RK, L.stage,
                               L.dts[tk.cs], nullptr, m.Q, m.mixed ? reinterpret_cast<T *>(m.Qc) : nullptr, m.Un,
                               reinterpret_cast<T *>(m.Unc), m.acc, &L.sync->nonfinite, c.ph);
      break;
    case TASK_CORRECT:
      correct_body<N, T>(tk.begin + threadIdx.x < tk.end ? tk.begin + threadIdx.x : (int64_t)1 << 62, Rpart, FI, m.ef,
                         met, m.E, MODE_RK, L.stage, L.dts[tk.cs], nullptr, m.Q,
                         m.mixed ? reinterpret_cast<T *>(m.Qc) : nullptr, m.Un, reinterpret_cast<T *>(m.Unc), m.acc,
                         &L.sync->nonfinite, c.ph);
      break;
  }
}

template <typename T, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1) k_batch_stage(BatchLaunch L) {
  extern __shared__ double smem[];
  __shared__ int s_task;
  if (L.debug_skip_block == (int)blockIdx.x) return;     // never arrives: the others time out
  for (int ph = 0; ph < L.n_phases; ++ph) {
    if (ph > 0 && !batch_grid_sync(L.sync, L.spin_limit)) return;
    const int t0 = L.phase_begin[ph], t1 = L.phase_begin[ph + 1];
    while (true) {
      __syncthreads();
      if (threadIdx.x == 0) s_task = t0 + (int)atomicAdd(&L.sync->counters[ph], 1u);
      __syncthreads();
      const int ti = s_task;
      if (ti >= t1) break;
      const BatchTask tk = L.tasks[ti];
      const BatchCase &c = L.cases[tk.cs];
      switch (c.m.N) {
        case 2: batch_task<T, 2>(tk, c, L, smem); break;
        case 3: batch_task<T, 3>(tk, c, L, smem); break;
        case 4: batch_task<T, 4>(tk, c, L, smem); break;
        case 5: batch_task<T, 5>(tk, c, L, smem); break;
        case 6: batch_task<T, 6>(tk, c, L, smem); break;
        case 7: if (BLOCK >= 352) batch_task<T, 7>(tk, c, L, smem); break;
        case 8: if (BLOCK >= 512) batch_task<T, 8>(tk, c, L, smem); break;
      }
    }
  }
}

}  // namespace
}  // namespace frx
