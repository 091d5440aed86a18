// Device bodies of the FR residual on the prisms of mixed hexahedral/prismatic meshes (arXiv 2308.06605,
// section "FR Algorithm", Eq. 1-3; the paper's solver handles prisms alongside hexahedra).
//
// A prism of order p carries Nt = N(N+1)/2 triangle nodes times N = p + 1 Gauss-Legendre points
// along its axis, point index m = q + Nt k.  With reference normals N_f (faces 0/1: zeta = -1/+1,
// triangles whose flux points are the triangle nodes; faces 2/3/4: s = -1, r + s = 0, r = -1,
// quadrilaterals with N x N Gauss points in (edge parameter, zeta)), the DG-equivalent correction
// (c = 0) is the lifting C_f = M^-1 E_f with the exact mass matrix, which factorises:
//   triangles:       C_f = h_-/+ (x) I_Nt        (h = the 1D correction divergence of the line)
//   quadrilaterals:  C_f = I_N (x) LQ_e,  LQ_e = M_T^-1 E_e^T diag(w)   (e = f - 2)
// and the traces are L_f = l(-1/+1) (x) I_Nt, resp. I_N (x) E_e (triangle interpolation to the
// edge's Gauss points).  The residual is R = -|J|^-1 [sum_d D~_d F^_d + sum_f C_f F^I_f] with the
// own-flux part of the correction folded into D~ (Drt, Dst, D1t of the operator table); BR2 uses
// grad Q = J^-T (D Q + sum_f N_f C_f (Q^I - Q_f)) and face gradients L_f (grad_unc + eta r_f),
// r_f = J^-T N_f C_f (Q^I - Q_f).  Interfaces, boundary states, common fluxes and the RK update
// are shared with the hexahedra (slot stride N^2; a triangular interface uses its first Nt slots).
//
// Templated on the order and on the element arithmetic T (double, or df32 on the mixed path),
// like the hexahedral kernels.
//
// The bodies are shared by the per-mesh prism kernels (fr_prism.cu) and the batched persistent
// stage kernel (fr_batch_kernel.cu); everything here has internal linkage.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "df32.cuh"
#include "fr_device.hpp"
#include "fr_point.cuh"

namespace frx {
namespace {


template <int N>
__host__ __device__ constexpr int prism_points() { return N * (N + 1) / 2 * N; }
template <int N>
__host__ __device__ constexpr int prism_threads() { return ((prism_points<N>() + 31) / 32) * 32; }
// Resident blocks the register budget must allow, per order and arithmetic (checked with ptxas):
// up to 64 threads, for double-float at 96 threads and at 128 threads (p = 5) about 170
// registers per thread without spills; FP64 at 96 threads fits 4 blocks unbounded; the larger
// blocks are bound by shared memory.
template <int N, typename T>
__host__ __device__ constexpr int prism_min_blocks() {
  return prism_threads<N>() <= 32 ? 12 : (prism_threads<N>() <= 64 ? 6 :
         (prism_threads<N>() <= 96 ? (std::is_same<T, df32>::value ? 4 : 2) : (prism_threads<N>() <= 128 ? 3 : 1)));
}
// Shared-memory values (of T) of the volume kernel: Q 5, grad 15, flux 15, BR2 weights 15, quad
// lifts 15 (per point) and the jumps of 5 faces x 5 variables x N^2 slots.
template <int N>
__host__ __device__ constexpr int prism_smem_values() { return 65 * prism_points<N>() + 25 * N * N; }


// Interface slot of local flux point r of prism face f for a packed face word.
template <int N>
__device__ __forceinline__ int prism_slot(int f, int r, int code, const int32_t *__restrict__ tri_slot) {
  constexpr int Nt = N * (N + 1) / 2;
  return f < 2 ? tri_slot[code * Nt + r] : orient_slot(code, r % N, r / N, N);
}

// ------------------------------------------------------------------------------------------
// 1. Solution traces.  Thread per (prism, face, flux point); triangular faces use r < Nt.
// ------------------------------------------------------------------------------------------
template <int N, typename T>
__device__ __forceinline__ void prism_interp_body(int64_t t, const T *__restrict__ Q, const int32_t *__restrict__ ef_p,
                                                  const T *__restrict__ tab, const int32_t *__restrict__ tri_slot,
                                                  T *__restrict__ Qtr, int64_t Ep) {
  constexpr int Nt = N * (N + 1) / 2, Np = Nt * N, Nf = N * N;
  constexpr PrismTab L = prism_tab(N);
  if (t >= Ep * 5 * Nf) return;
  const int r = (int)(t % Nf);
  const int64_t eff = t / Nf;
  const int f = (int)(eff % 5);
  const int64_t e = eff / 5;
  if (f < 2 && r >= Nt) return;
  const T *q = Q + e * Np * 5;
  Dot<T> acc[5];
  if (f < 2) {
    const T *l = tab + (f ? L.lp : L.lm);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const T lk = l[k];
      const T *qk = q + (r + Nt * k) * 5;
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v].add(lk, qk[v]);
    }
  } else {
    const int a = r % N, b = r / N;
    const T *Ea = tab + L.E + (f - 2) * N * Nt + a * Nt;
#pragma unroll 4
    for (int j = 0; j < Nt; ++j) {
      const T ej = Ea[j];
      const T *qj = q + (j + Nt * b) * 5;
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v].add(ej, qj[v]);
    }
  }
  const int packed = ef_p[eff];
  const int64_t I = packed >> 4;
  const int side = (packed >> 3) & 1;
  T *dst = Qtr + (I * 2 + side) * 5 * Nf + prism_slot<N>(f, r, packed & 7, tri_slot);
#pragma unroll
  for (int v = 0; v < 5; ++v) dst[v * Nf] = acc[v].get();
}

// ------------------------------------------------------------------------------------------
// 2. Volume kernel.  One block per prism, one thread per solution point.
// ------------------------------------------------------------------------------------------
// One prism e handled by `nth` threads of the block (thread index tid in [0, nth)); every thread
// of the block calls this together (it contains block barriers); inactive sub-blocks
// (active = false) only take part in the barriers.
template <int N, typename T>
__device__ __forceinline__ void prism_volume_body(int64_t e, int tid, int nth, bool active, double *sm_raw,
                                                  const T *__restrict__ Q, const T *__restrict__ metrics,
                                                  const int32_t *__restrict__ ef_p, const T *__restrict__ Qtr,
                                                  const T *__restrict__ tab, const int32_t *__restrict__ tri_slot,
                                                  T *__restrict__ Gtr, T *__restrict__ Rpart, const DevPhys &dph,
                                                  const int8_t *__restrict__ if_up, int64_t n_interior) {
  constexpr int Nt = N * (N + 1) / 2, Np = Nt * N, Nf = N * N;
  constexpr PrismTab L = prism_tab(N);
  T *sm = reinterpret_cast<T *>(sm_raw);
  T *sQ = sm;                 // [5][Np]
  T *sG = sQ + 5 * Np;        // [15][Np] uncorrected physical gradient, index j*5+v
  T *sH = sG + 15 * Np;       // [15][Np] transformed flux, index d*5+v
  T *sW = sH + 15 * Np;       // [5][3][Np] eta (N_f . S[.][j]) / |J|: BR2 lifting to physical space
  T *sL = sW + 15 * Np;       // [3][5][Np] C_f (Q^I - Q_f) of the quadrilateral faces
  T *sdQ = sL + 15 * Np;      // [5][5][Nf] Q^I - Q_own at the flux points
  const PhysT<T> &ph = phys_of<T>(dph);
  const bool viscous = dph.viscous != 0;
  if (active)
    for (int t = tid; t < 5 * Np; t += nth) sQ[(t % 5) * Np + t / 5] = Q[e * Np * 5 + t];
  if (viscous && active) {
    for (int t = tid; t < 5 * Nf; t += nth) {
      const int f = t / Nf, r = t % Nf;
      if (f < 2 && r >= Nt) continue;
      const int packed = ef_p[e * 5 + f];
      const int64_t I = packed >> 4;
      const int side = (packed >> 3) & 1;
      const int slot = prism_slot<N>(f, r, packed & 7, tri_slot);
      const T *own = Qtr + (I * 2 + side) * 5 * Nf + slot;
      const T *oth = Qtr + (I * 2 + (1 - side)) * 5 * Nf + slot;
      // Q^I - Q_own: BR2 (other - own)/2; LDG 0 on the supplying side, other - own on the other.
      T w = ph.half;
      if (dph.ldg && I < n_interior) w = side == (if_up[I] ? 0 : 1) ? ph.zero : ph.one;
#pragma unroll
      for (int v = 0; v < 5; ++v) sdQ[(f * 5 + v) * Nf + r] = w * (oth[v * Nf] - own[v * Nf]);
    }
  }
  __syncthreads();
  const bool pt = active && tid < Np;
  const int m = tid < Np ? tid : 0, q = m % Nt, k = m / Nt;
  if (pt) {
    T S[9], invJ, qv[5], G[15];
    const T *met = metrics + e * 10 * Np + m;
#pragma unroll
    for (int c = 0; c < 9; ++c) S[c] = met[c * Np];
    invJ = met[9 * Np];
#pragma unroll
    for (int v = 0; v < 5; ++v) qv[v] = sQ[v * Np + m];
    if (viscous) {
      const T *Dr = tab + L.Dr + q * Nt, *Ds = tab + L.Ds + q * Nt, *D1 = tab + L.D1 + k * N;
      const T hmk = tab[L.hm + k], hpk = tab[L.hp + k];
      const T *LQ0 = tab + L.LQ + q * N, *LQ1 = LQ0 + Nt * N, *LQ2 = LQ1 + Nt * N;
      T sj[9];   // S[d][jj] / |J|
#pragma unroll
      for (int c = 0; c < 9; ++c) sj[c] = S[c] * invJ;
      // One variable at a time: reference gradient, liftings, correction, physical transform.  The
      // loop stays rolled (a smaller instruction footprint): the corrected gradient goes through this
      // thread's own entries of the transformed-flux buffer, which only this thread writes later.
#pragma unroll 1
      for (int v = 0; v < 5; ++v) {
        const T *sq = sQ + v * Np;
        Dot<T> a0, a1, a2;
#pragma unroll 4
        for (int j = 0; j < Nt; ++j) {
          const T qj = sq[j + Nt * k];
          a0.add(Dr[j], qj);
          a1.add(Ds[j], qj);
        }
#pragma unroll
        for (int c = 0; c < N; ++c) a2.add(D1[c], sq[q + Nt * c]);
        const T gu0 = a0.raw(), gu1 = a1.raw(), gu2 = a2.raw();
        // Lifted jumps: quadrilateral faces (edge e = f - 2) and the two triangles.
        Dot<T> l2, l3, l4;
#pragma unroll
        for (int a = 0; a < N; ++a) {
          l2.add(LQ0[a], sdQ[(2 * 5 + v) * Nf + a + N * k]);
          l3.add(LQ1[a], sdQ[(3 * 5 + v) * Nf + a + N * k]);
          l4.add(LQ2[a], sdQ[(4 * 5 + v) * Nf + a + N * k]);
        }
        const T L2 = l2.raw(), L3 = l3.raw(), L4 = l4.raw();
        sL[(0 * 5 + v) * Np + m] = L2;
        sL[(1 * 5 + v) * Np + m] = L3;
        sL[(2 * 5 + v) * Np + m] = L4;
        // sum_f N_f C_f dQ_f with N = (0,0,-1), (0,0,1), (0,-1,0), (1,1,0), (-1,0,0).
        a0.add(ph.one, L3);
        a0.add(-ph.one, L4);
        a1.add(-ph.one, L2);
        a1.add(ph.one, L3);
        a2.add(-hmk, sdQ[(0 * 5 + v) * Nf + q]);
        a2.add(hpk, sdQ[(1 * 5 + v) * Nf + q]);
        const T gc0 = a0.raw(), gc1 = a1.raw(), gc2 = a2.raw();
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
          Dot<T> du, dc;
          du.add(sj[0 * 3 + jj], gu0);
          du.add(sj[1 * 3 + jj], gu1);
          du.add(sj[2 * 3 + jj], gu2);
          dc.add(sj[0 * 3 + jj], gc0);
          dc.add(sj[1 * 3 + jj], gc1);
          dc.add(sj[2 * 3 + jj], gc2);
          const T gc = dc.raw();
          sH[(jj * 5 + v) * Np + m] = gc;
          sG[(jj * 5 + v) * Np + m] = dph.ldg ? gc : du.raw();   // LDG: corrected
        }
      }
#pragma unroll
      for (int c = 0; c < 15; ++c) G[c] = sH[c * Np + m];
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) {
        const T ej = ph.eta * invJ;
        sW[(0 * 3 + jj) * Np + m] = -(ej * S[2 * 3 + jj]);
        sW[(1 * 3 + jj) * Np + m] = ej * S[2 * 3 + jj];
        sW[(2 * 3 + jj) * Np + m] = -(ej * S[1 * 3 + jj]);
        sW[(3 * 3 + jj) * Np + m] = ej * (S[0 * 3 + jj] + S[1 * 3 + jj]);
        sW[(4 * 3 + jj) * Np + m] = -(ej * S[0 * 3 + jj]);
      }
    }
    {
      // Transformed fluxes per reference direction from the contravariant velocity.
      const T ri = ph.one / qv[0];
      const T u[3] = {qv[1] * ri, qv[2] * ri, qv[3] * ri};
      const T p = ph.gm1 * (qv[4] - ph.half * (qv[1] * u[0] + qv[2] * u[1] + qv[3] * u[2]));
      T tau[3][3], hq[3];
      if (viscous) viscous_stress<T>(qv, u, ri, G, ph, visc_of(ph), tau, hq);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        T f[5];
        contravariant_flux<T>(qv, u, p, S + 3 * d, viscous, tau, hq, f);
#pragma unroll
        for (int v = 0; v < 5; ++v) sH[(d * 5 + v) * Np + m] = f[v];
      }
    }
  }
  __syncthreads();
  if (viscous && active) {
    // Gradient traces: interpolated uncorrected gradient + eta * own lifting.  One item per
    // (gradient component jj, face point) keeps the block busy.
    for (int t = tid; t < 15 * Nf; t += nth) {
      const int jj = t / (5 * Nf), fr_ = t - jj * 5 * Nf;
      const int f = fr_ / Nf, r = fr_ % Nf;
      if (f < 2 && r >= Nt) continue;
      const int packed = ef_p[e * 5 + f];
      const int64_t I = packed >> 4;
      const int side = (packed >> 3) & 1;
      T *dst = Gtr + (I * 2 + side) * 15 * Nf + prism_slot<N>(f, r, packed & 7, tri_slot);
      if (f < 2) {
        const T *l = tab + (f ? L.lp : L.lm), *hh = tab + (f ? L.hp : L.hm);
        Dot<T> lf;
#pragma unroll
        for (int c = 0; c < N; ++c) lf.add(l[c] * hh[c], sW[(f * 3 + jj) * Np + r + Nt * c]);
        const T lfac = lf.raw();
#pragma unroll 1
        for (int v = 0; v < 5; ++v) {
          Dot<T> acc;
#pragma unroll
          for (int c = 0; c < N; ++c) acc.add(l[c], sG[(jj * 5 + v) * Np + r + Nt * c]);
          acc.add(lfac, sdQ[(f * 5 + v) * Nf + r]);
          dst[(jj * 5 + v) * Nf] = acc.raw();
        }
      } else {
        const int a = r % N, b = r / N;
        const T *Ea = tab + L.E + (f - 2) * N * Nt + a * Nt;
        const T *lq = sL + ((f - 2) * 5) * Np + Nt * b;
        const T *w = sW + (f * 3 + jj) * Np + Nt * b;
#pragma unroll 1
        for (int v = 0; v < 5; ++v) {
          const T *g = sG + (jj * 5 + v) * Np + Nt * b;
          Dot<T> acc;
          for (int j = 0; j < Nt; ++j) {
            acc.add(Ea[j], g[j]);
            acc.add(Ea[j] * w[j], lq[v * Np + j]);
          }
          dst[(jj * 5 + v) * Nf] = acc.raw();
        }
      }
    }
  }
  if (pt) {
    const T *Drt = tab + L.Drt + q * Nt, *Dst = tab + L.Dst + q * Nt, *D1t = tab + L.D1t + k * N;
    T *out = Rpart + (e * Np + m) * 5;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const T *h0 = sH + (0 * 5 + v) * Np + Nt * k, *h1 = sH + (1 * 5 + v) * Np + Nt * k;
      const T *h2 = sH + (2 * 5 + v) * Np + q;
      Dot<T> acc;
#pragma unroll 4
      for (int j = 0; j < Nt; ++j) {
        acc.add(Drt[j], h0[j]);
        acc.add(Dst[j], h1[j]);
      }
#pragma unroll
      for (int c = 0; c < N; ++c) acc.add(D1t[c], h2[Nt * c]);
      out[v] = acc.raw();
    }
  }
}

// ------------------------------------------------------------------------------------------
// 4. Correction by the common flux, scaling and output / RK44 update.  Thread per prism point.
// ------------------------------------------------------------------------------------------
template <int N, typename T>
__device__ __forceinline__ void prism_correct_body(int64_t t, const T *__restrict__ Rpart, const T *__restrict__ FI,
                                                   const int32_t *__restrict__ ef_p, const T *__restrict__ metrics,
                                                   const T *__restrict__ tab, const int32_t *__restrict__ tri_slot,
                                                   int64_t Ep, int64_t first_point, int mode, int stage, double dt,
                                                   double *__restrict__ Rout, double *__restrict__ Q,
                                                   T *__restrict__ Qc, double *__restrict__ Un, T *__restrict__ Unc,
                                                   double *__restrict__ acc, int *__restrict__ flag,
                                                   const DevPhys &dph) {
  constexpr int Nt = N * (N + 1) / 2, Np = Nt * N, Nf = N * N;
  constexpr PrismTab L = prism_tab(N);
  if (t >= Ep * Np) return;
  const int64_t e = t / Np;
  const int m = (int)(t % Np), q = m % Nt, k = m / Nt;
  const PhysT<T> &ph = phys_of<T>(dph);
  Dot<T> r[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) r[v].add(ph.one, Rpart[t * 5 + v]);
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    const int packed = ef_p[e * 5 + f];
    const int64_t I = packed >> 4;
    const int side = (packed >> 3) & 1;
    const T h = tab[(f ? L.hp : L.hm) + k];
    const T w = side ? -h : h;
    const T *src = FI + I * 5 * Nf + tri_slot[(packed & 7) * Nt + q];
#pragma unroll
    for (int v = 0; v < 5; ++v) r[v].add(w, src[v * Nf]);
  }
#pragma unroll
  for (int f = 2; f < 5; ++f) {
    const int packed = ef_p[e * 5 + f];
    const int64_t I = packed >> 4;
    const int side = (packed >> 3) & 1;
    const T *lq = tab + L.LQ + (f - 2) * Nt * N + q * N;
    const T *src = FI + I * 5 * Nf;
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const T w = side ? -lq[a] : lq[a];
      const int slot = orient_slot(packed & 7, a, k, N);
#pragma unroll
      for (int v = 0; v < 5; ++v) r[v].add(w, src[v * Nf + slot]);
    }
  }
  const T s = -metrics[(e * 10 + 9) * Np + m];
  T rv[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) rv[v] = r[v].get();
  finish_point<T>(first_point + t, rv, s, mode, stage, dt, Rout, Q, Qc, Un, Unc, acc, flag, dph);
}

}  // namespace
}  // namespace frx
