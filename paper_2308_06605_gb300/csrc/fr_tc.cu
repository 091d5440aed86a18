// Face interpolation (section "FR Algorithm", Eq. 2: the solution at the flux points of each face,
// Q_f = sum_a l_a(+-1) Q_a along the face's normal line) on the tensor cores, for the
// double-float element arithmetic (FR_PREC_MIXED_TC).
//
// The contraction of every line of N solution values with the two boundary-value vectors l(-1),
// l(+1) is done by tcgen05.mma in TF32 with FP32 accumulation, made exact by splitting both
// operands into exponent-aligned slices (the error-free splitting of Ozaki, Ogita, Oishi & Rump,
// "Error-free transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012):
//   * a line x_a (double-float hi + lo) with sigma = 2^E > max |x| is written as
//     x = sigma sum_{s=0..4} 2^{-beta (s+1)} X_s + O(2^{-5 beta} sigma), beta = 10, where every X_s is
//     an integer with |X_0| <= 2^beta, |X_s| <= 2^{beta-1} (round-to-nearest slicing), exactly
//     representable in TF32;
//   * each operator row (l(-1) or l(+1)) likewise with its own tau = 2^F > max |l|, slices O_t;
//   * one MMA per data slice s multiplies the 128 lines' X_s (A, 128 x 8) with all operator slices
//     at once (B, 16 x 8: row 2t + j = slice t of operator row j), so D_s[r][2t + j] =
//     sum_a X_s[r][a] O_t[j][a]: integers below 8 * 2^{2 beta} = 2^23, hence exact in the FP32
//     accumulator whatever the order of its additions;
//   * per output the level sums A_L = sum_{s+t=L} D_s (L = 0..4; exact below 2^24 for L <= 3,
//     the last level's rounding is 2^{-24} of a 2^{-40} term) are combined into a double-float
//     value, sum_L 2^{-beta L} A_L, scaled by sigma tau 2^{-2 beta}.
// Dropped terms (s + t > 4) and the last slice's rounding leave 2^{-51} sigma tau per output; the
// double-float result's own rounding (48 bits of a value up to 8 sigma tau) brings the total to at
// most 2^{-44} sigma tau.  (With four slices, 2^{-41}, the error of a Ma 0.1 continuity residual
// reached 1e-6 of its largest entry: the trace jump is amplified by the Rusanov dissipation.)
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "df32.cuh"
#include "fr_device.hpp"
#include "tc05.cuh"

namespace frx {
namespace {

constexpr int kBeta = 10;
constexpr int kSlices = 5;
constexpr int kTcThreads = 128;
constexpr int kTmemCols = 128;                   // 5 accumulators of 16 columns, rounded to a power of 2
constexpr long long kWaitLimit = 4000000000ll;   // clock cycles (about 2 s) before a wait gives up

// Operator slices per order (index N - 1): the B tile of 16 rows x K = 8 in the K-major core-matrix
// layout (512 bytes), and the row scales tau_j (j = 0: l(-1), 1: l(+1)).
__device__ __align__(128) float g_tc_ops[kMaxN][128];
__constant__ float c_tc_tau[kMaxN][2];

}  // namespace

// Host: slices of the boundary-value vectors of every order, by the same round-to-nearest
// splitting as the device applies to the data.
cudaError_t upload_tc_tables() {
  float ops[kMaxN][128];
  float tau[kMaxN][2];
  std::memset(ops, 0, sizeof ops);
  std::memset(tau, 0, sizeof tau);
  for (int p = 1; p < kMaxN; ++p) {
    const Basis1D b = make_basis(p);
    const int N = b.N;
    for (int j = 0; j < 2; ++j) {
      const double *row = j == 0 ? b.lm : b.lp;
      double mx = 0.0;
      for (int a = 0; a < N; ++a) mx = std::fmax(mx, std::fabs(row[a]));
      int F = 0;
      std::frexp(mx, &F);                       // mx < 2^F
      tau[N - 1][j] = (float)std::ldexp(1.0, F);
      for (int a = 0; a < N; ++a) {
        double y = std::ldexp(row[a], -F);
        for (int t = 0; t < kSlices; ++t) {
          const double u = std::ldexp(y, kBeta);
          const double s = std::nearbyint(u);
          y = u - s;
          const int n = 2 * t + j;
          ops[N - 1][tc::kmajor_off(n, a) / 4] = (float)s;
        }
      }
    }
  }
  cudaError_t e = cudaMemcpyToSymbol(g_tc_ops, ops, sizeof ops);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tc_tau, tau, sizeof tau);
  return e;
}

namespace {

// Flux point r = a + N b of a face normal to axis d: base index of its normal line and the stride
// along it (point index m = i + N j + N^2 k; the face's two tangential axes, lower first).
template <int N>
__device__ __forceinline__ void line_of(int d, int r, int &base, int &sd) {
  const int t0 = (d == 0) ? 1 : 0, t1 = (d == 2) ? 1 : 2;
  const int a = r % N, b = r / N;
  const int st[3] = {1, N, N * N};
  base = a * st[t0] + b * st[t1];
  sd = st[d];
}

__device__ __forceinline__ int slot_in(int code, int a, int b, int N) {
  if (code & 4) { int t = a; a = b; b = t; }
  if (code & 1) a = N - 1 - a;
  if (code & 2) b = N - 1 - b;
  return a + N * b;
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }   // -126 <= e <= 127

// One CTA of 128 threads handles 128 consecutive lines of the global line list (element e, then
// direction d, variable v, face point t: line g = e 15 N^2 + (5 d + v) N^2 + t); thread r owns line
// r of the tile: it gathers and slices its N values, and after the MMAs reads its own TMEM lane.
template <int N>
__global__ void __launch_bounds__(kTcThreads) k_interp_tc(const df32 *__restrict__ Q, const int32_t *__restrict__ ef,
                                                          df32 *__restrict__ Qtr, int64_t E, int *__restrict__ err) {
  constexpr int Np = N * N * N, Nf = N * N, L = 15 * Nf;
  __shared__ __align__(1024) float sA[kSlices][kTcThreads * 8];
  __shared__ __align__(128) float sB[128];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tbase;
  __shared__ int s_issued;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t g = (int64_t)blockIdx.x * kTcThreads + tid;
  const bool live = g < E * L;
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
    s_issued = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(&tbase, kTmemCols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid == 0) {
    tc::mbar_arrive_expect_tx(&bar, 512);
    tc::bulk_g2s(sB, &g_tc_ops[N - 1][0], 512, &bar);
  }
  // Gather the line and split it into exponent-aligned slices.
  float X[kSlices][N];
  int64_t e = 0;
  int d = 0, v = 0, t = 0, Ex = 0;
  bool nonzero = false;
  if (live) {
    e = g / L;
    const int l = (int)(g - e * L);
    const int dv = l / Nf;
    t = l - dv * Nf;
    d = dv / 5;
    v = dv - 5 * d;
    int base, sd;
    line_of<N>(d, t, base, sd);
    df32 x[N];
    float mx = 0.f;
#pragma unroll
    for (int a = 0; a < N; ++a) {
      x[a] = Q[(e * Np + base + a * sd) * 5 + v];
      mx = fmaxf(mx, fabsf(x[a].hi));
    }
    nonzero = mx > 0.f;
    if (nonzero) {
      frexpf(mx, &Ex);                     // mx < 2^Ex
      Ex = max(min(Ex, 90), -90);           // keeps every power of two below in range
    }
    const float sc = pow2f(kBeta - Ex), sc_lo = pow2f(3 * kBeta - Ex), up = pow2f(kBeta);
#pragma unroll
    for (int a = 0; a < N; ++a) {
      float u = x[a].hi * sc;
      X[0][a] = rintf(u);
      u = (u - X[0][a]) * up;
      X[1][a] = rintf(u);
      // hi's remaining bits plus lo, kept exact as a pair: the third slice rounds their sum and
      // the pair's rounding error is carried into the next remainder.
      const df32 w = two_sum((u - X[1][a]) * up, x[a].lo * sc_lo);
      X[2][a] = rintf(w.hi);
      u = ((w.hi - X[2][a]) + w.lo) * up;
      X[3][a] = rintf(u);
      u = (u - X[3][a]) * up;
      X[4][a] = rintf(u);
      if (!nonzero) X[0][a] = X[1][a] = X[2][a] = X[3][a] = X[4][a] = 0.f;
    }
  }
#pragma unroll
  for (int s = 0; s < kSlices; ++s)
#pragma unroll
    for (int k = 0; k < 8; ++k) sA[s][tc::kmajor_off(tid, k) / 4] = (live && k < N) ? X[s][k] : 0.f;
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0) {
    tc::fence_after_sync();
    if (tc::mbar_wait(&bar, 0, kWaitLimit)) {
      const uint64_t bdesc = tc::smem_desc(sB, 128, 256);
      constexpr uint32_t idesc = tc::idesc_tf32(128, 16);
#pragma unroll
      for (int s = 0; s < kSlices; ++s)
        tc::mma_tf32(tbase + 16 * s, tc::smem_desc(&sA[s][0], 128, 256), bdesc, idesc, 0);
      tc::mma_commit(&bar);
      s_issued = 1;
    } else {
      atomicOr(err, 2);
    }
  }
  __syncthreads();
  const bool issued = s_issued != 0;
  bool done = issued && tc::mbar_wait(&bar, 1, kWaitLimit);
  done = __syncthreads_and(done) != 0;
  tc::fence_after_sync();
  if (issued && !done) {
    if (tid == 0) atomicOr(err, 2);
    // The MMAs may still be writing TMEM: wait once more (bounded) before releasing it.
    tc::mbar_wait(&bar, 1, kWaitLimit);
  }
  if (done) {
    // Columns 2t + j of D_s for s + t <= 4: 10 columns of D_0, 8 of the others.
    const uint32_t lane = (uint32_t)(warp * 32) << 16;
    float D0[16], D[kSlices][8];
    tc::tmem_ld16(tbase + lane, D0);
#pragma unroll
    for (int s = 1; s < kSlices; ++s) tc::tmem_ld8(tbase + lane + 16 * s, D[s]);
    tc::tmem_ld_wait();
#pragma unroll
    for (int c = 0; c < 8; ++c) D[0][c] = D0[c];
    if (live) {
      const float sigma = pow2f(Ex), m10 = pow2f(-kBeta), m20 = pow2f(-2 * kBeta), m30 = pow2f(-3 * kBeta),
                  m40 = pow2f(-4 * kBeta);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        // Level sums (exact: integers below 2^24), then sum_L 2^{-beta L} A_L as a double-float.
        const float A0 = D[0][j];
        const float A1 = D[0][2 + j] + D[1][j];
        const float A2 = D[0][4 + j] + D[1][2 + j] + D[2][j];
        const float A3 = D[0][6 + j] + D[1][4 + j] + D[2][2 + j] + D[3][j];
        const float A4 = D0[8 + j] + D[1][6 + j] + D[2][4 + j] + D[3][2 + j] + D[4][j];
        const df32 h = two_sum(A0, A1 * m10);
        const float lo = fmaf(A4, m40, fmaf(A3, m30, A2 * m20));
        df32 r = two_sum(h.hi, h.lo + lo);
        const float scale = sigma * c_tc_tau[N - 1][j] * m20;
        r.hi *= scale;
        r.lo *= scale;
        if (!nonzero) r = df(0.f, 0.f);
        const int packed = ef[e * 6 + 2 * d + j];
        const int64_t I = packed >> 4;
        const int side = (packed >> 3) & 1;
        Qtr[(I * 2 + side) * 5 * Nf + v * Nf + slot_in(packed & 7, t % N, t / N, N)] = r;
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, kTmemCols);
}

template <int N>
cudaError_t interp_tc_impl(const DevMesh &m, cudaStream_t st) {
  const int64_t lines = m.E * 15 * N * N;
  if (lines == 0) return cudaSuccess;
  k_interp_tc<N><<<(unsigned)((lines + kTcThreads - 1) / kTcThreads), kTcThreads, 0, st>>>(
      reinterpret_cast<const df32 *>(m.Qc), m.ef, reinterpret_cast<df32 *>(m.Qtr), m.E, m.flag);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_interp_tc(const DevMesh &m, cudaStream_t st) {
  switch (m.N) {
    case 2: return interp_tc_impl<2>(m, st);
    case 3: return interp_tc_impl<3>(m, st);
    case 4: return interp_tc_impl<4>(m, st);
    case 5: return interp_tc_impl<5>(m, st);
    case 6: return interp_tc_impl<6>(m, st);
    case 7: return interp_tc_impl<7>(m, st);
    case 8: return interp_tc_impl<8>(m, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace frx
