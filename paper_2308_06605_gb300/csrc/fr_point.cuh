// Pointwise device functions shared by the hexahedral and prismatic kernels: gas dynamics (normal
// inviscid flux with the Rusanov wave-speed bound, viscous flux with optional eddy viscosity) and
// the output / RK44 stage update of one solution point.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "df32.cuh"
#include "fr_device.hpp"

namespace frx {

template <typename T> __device__ __forceinline__ const PhysT<T> &phys_of(const DevPhys &p);
template <> __device__ __forceinline__ const PhysT<double> &phys_of<double>(const DevPhys &p) { return p.d; }
template <> __device__ __forceinline__ const PhysT<df32> &phys_of<df32>(const DevPhys &p) { return p.f; }
template <> __device__ __forceinline__ const PhysT<float> &phys_of<float>(const DevPhys &p) { return p.s; }

// ------------------------------------------------------------------------------------------
// Gas dynamics (ideal gas, Stokes hypothesis, constant mu, Fourier heat flux).
// ------------------------------------------------------------------------------------------
// Normal inviscid flux F(q).n and (|u.n^| + c)|n|, in FP64 (pressure/energy recovery); nn = |n|.
__device__ __forceinline__ void normal_inviscid(const double q[5], const double n[3], double nn, double g,
                                                double out[5], double &un_abs_plus_c_n) {
  const double ri = 1.0 / q[0];
  const double u = q[1] * ri, v = q[2] * ri, w = q[3] * ri;
  const double p = (g - 1.0) * (q[4] - 0.5 * (q[1] * u + q[2] * v + q[3] * w));
  const double un = u * n[0] + v * n[1] + w * n[2];
  out[0] = q[0] * un;
  out[1] = q[1] * un + p * n[0];
  out[2] = q[2] * un + p * n[1];
  out[3] = q[3] * un + p * n[2];
  out[4] = (q[4] + p) * un;
  un_abs_plus_c_n = fabs(un) + sqrt(g * p * ri) * nn;      // (|u.n^| + c) |n|
}

// Double-float normal flux with the pressure recovery p = (gamma-1)(E - m.u/2) in FP64.
__device__ __forceinline__ void normal_inviscid(const df32 q[5], const df32 n[3], df32 nn, const DevPhys &dph,
                                                df32 out[5], df32 &un_abs_plus_c_n) {
  const PhysT<df32> &ph = dph.f;
  const df32 ri = ph.one / q[0];
  const df32 u[3] = {q[1] * ri, q[2] * ri, q[3] * ri};
  Dot<df32> mu, unn;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    mu.add(q[1 + c], u[c]);
    unn.add(u[c], n[c]);
  }
  const double pd = (dph.gamma - 1.0) * (to_double(q[4]) - 0.5 * to_double(mu.get()));
  const df32 p = df_from(pd);
  const df32 un = unn.get();
  out[0] = q[0] * un;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Dot<df32> f;
    f.add(q[1 + c], un);
    f.add(p, n[c]);
    out[1 + c] = f.get();
  }
  out[4] = (q[4] + p) * un;
  un_abs_plus_c_n = fabs(un) + sqrt(ph.gamma * p * ri) * nn;
}

// FP64 overload with the same signature shape (the FP64 path's arithmetic).
__device__ __forceinline__ void normal_inviscid(const double q[5], const double n[3], double nn, const DevPhys &dph,
                                                double out[5], double &s) {
  normal_inviscid(q, n, nn, dph.gamma, out, s);
}

// Roe's approximate Riemann flux (Roe 1981) through the area-scaled normal n (|n| = nn), FP64:
// 1/2 (F(qL) + F(qR)).n - 1/2 |n| sum_k |lambda_k| alpha_k r_k over the waves of the Jacobian at the
// Roe average (density-weighted velocity and total enthalpy): acoustic waves u.n^ -/+ c with
// strengths (dp -/+ rho c du_n) / (2 c^2), entropy wave u.n^ with drho - dp / c^2, shear wave u.n^
// carrying rho (du - du_n n^).  Harten's entropy fix on the acoustic waves: |lambda| below
// d = 0.1 c becomes (lambda^2 + d^2) / (2 d).
__device__ __forceinline__ void roe_flux(const double qL[5], const double qR[5], const double n[3], double nn,
                                         double g, double F[5]) {
  double fL[5], fR[5], sL, sR;
  normal_inviscid(qL, n, nn, g, fL, sL);
  normal_inviscid(qR, n, nn, g, fR, sR);
  const double inn = 1.0 / nn;
  const double nh[3] = {n[0] * inn, n[1] * inn, n[2] * inn};
  const double rL = qL[0], rR = qR[0];
  const double uL[3] = {qL[1] / rL, qL[2] / rL, qL[3] / rL}, uR[3] = {qR[1] / rR, qR[2] / rR, qR[3] / rR};
  const double pL = (g - 1.0) * (qL[4] - 0.5 * (qL[1] * uL[0] + qL[2] * uL[1] + qL[3] * uL[2]));
  const double pR = (g - 1.0) * (qR[4] - 0.5 * (qR[1] * uR[0] + qR[2] * uR[1] + qR[3] * uR[2]));
  const double HL = (qL[4] + pL) / rL, HR = (qR[4] + pR) / rR;
  const double sl = sqrt(rL), sr = sqrt(rR), w = 1.0 / (sl + sr);
  const double r = sl * sr;
  double u[3], du[3], q2 = 0.0, un = 0.0, dun = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    u[c] = (sl * uL[c] + sr * uR[c]) * w;
    du[c] = uR[c] - uL[c];
    q2 += u[c] * u[c];
    un += u[c] * nh[c];
    dun += du[c] * nh[c];
  }
  const double H = (sl * HL + sr * HR) * w;
  const double c2 = (g - 1.0) * (H - 0.5 * q2), c = sqrt(c2);
  const double dp = pR - pL, dr = rR - rL;
  const double a1 = (dp - r * c * dun) / (2.0 * c2), a2 = dr - dp / c2, a3 = (dp + r * c * dun) / (2.0 * c2);
  const double d = 0.1 * c;
  auto fix = [d](double lam) {
    const double a = fabs(lam);
    return a < d ? (lam * lam + d * d) / (2.0 * d) : a;
  };
  const double l1 = fix(un - c) * a1, l2 = fabs(un), l3 = fix(un + c) * a3;
  double sh[3], ush = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    sh[k] = r * (du[k] - dun * nh[k]);
    ush += u[k] * sh[k];
  }
  double D[5];
  D[0] = l1 + l2 * a2 + l3;
#pragma unroll
  for (int k = 0; k < 3; ++k) D[1 + k] = l1 * (u[k] - c * nh[k]) + l3 * (u[k] + c * nh[k]) + l2 * (a2 * u[k] + sh[k]);
  D[4] = l1 * (H - c * un) + l3 * (H + c * un) + l2 * (a2 * 0.5 * q2 + ush);
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * nn * D[v];
}

// Transport coefficients of one viscous-flux evaluation (molecular, or with an eddy viscosity).
template <typename T>
struct Visc {
  T mu, m2mu3, kappa;   // mu, -2 mu / 3, kappa
};

template <typename T>
__device__ __forceinline__ Visc<T> visc_of(const PhysT<T> &ph) {
  return Visc<T>{ph.mu, ph.m2mu3, ph.kappa};
}

// Closure: mu + rho nu_t, kappa + rho nu_t cp / Pr_t (nu_t = 0 gives the molecular values exactly).
template <typename T>
__device__ __forceinline__ Visc<T> visc_with(const PhysT<T> &ph, T rho_nu, const DevPhys &dph) {
  if (!dph.closure) return visc_of(ph);
  const T mu = ph.mu + rho_nu;
  return Visc<T>{mu, ph.m2mu3 + from_double<T>(-2.0 / 3.0) * rho_nu, ph.kappa + from_double<T>(dph.cp_prt) * rho_nu};
}

// Viscous flux F_v[j][v] (j = direction) of state q with gradient G[j*5 + v] = dQ_v/dx_j.
template <typename T>
__device__ __forceinline__ void viscous_flux(const T q[5], const T *G, const PhysT<T> &ph, const Visc<T> &vc,
                                             T Fv[3][5]) {
  const T ri = ph.one / q[0];
  const T u[3] = {q[1] * ri, q[2] * ri, q[3] * ri};
  const T eo = q[4] * ri;
  T du[3][3];   // du[i][j] = du_i/dx_j
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) du[i][j] = (G[j * 5 + 1 + i] - u[i] * G[j * 5]) * ri;
  T dT[3];
#pragma unroll
  for (int j = 0; j < 3; ++j)
    dT[j] = ph.cT * ((G[j * 5 + 4] - eo * G[j * 5]) * ri - (u[0] * du[0][j] + u[1] * du[1][j] + u[2] * du[2][j]));
  const T lam = vc.m2mu3 * (du[0][0] + du[1][1] + du[2][2]);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    T t[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      t[i] = vc.mu * (du[i][j] + du[j][i]);
      if (i == j) t[i] = t[i] + lam;
    }
    Fv[j][0] = ph.zero;
    Fv[j][1] = t[0];
    Fv[j][2] = t[1];
    Fv[j][3] = t[2];
    Fv[j][4] = u[0] * t[0] + u[1] * t[1] + u[2] * t[2] + vc.kappa * dT[j];
  }
}

// Viscous stress tau[i][j] = mu (du_i/dx_j + du_j/dx_i) + delta_ij lambda div u and heat-flux
// term hq[j] = kappa dT/dx_j of state q with gradient G[j*5 + v] = dQ_v/dx_j (the entries of
// viscous_flux: Fv[j][1+i] = tau[i][j], Fv[j][4] = sum_i u_i tau[i][j] + hq[j]).
template <typename T>
__device__ __forceinline__ void viscous_stress(const T q[5], const T u[3], T ri, const T *G, const PhysT<T> &ph,
                                               const Visc<T> &vc, T tau[3][3], T hq[3]) {
  const T eo = q[4] * ri;
  T du[3][3];   // du[i][j] = du_i/dx_j
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) du[i][j] = (G[j * 5 + 1 + i] - u[i] * G[j * 5]) * ri;
#pragma unroll
  for (int j = 0; j < 3; ++j)
    hq[j] = vc.kappa * (ph.cT * ((G[j * 5 + 4] - eo * G[j * 5]) * ri -
                                 (u[0] * du[0][j] + u[1] * du[1][j] + u[2] * du[2][j])));
  const T lam = vc.m2mu3 * (du[0][0] + du[1][1] + du[2][2]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      tau[i][j] = vc.mu * (du[i][j] + du[j][i]);
      if (i == j) tau[i][j] = tau[i][j] + lam;
      tau[j][i] = tau[i][j];
    }
}

// Transformed flux of reference direction d, F^_d = sum_j S[d][j] (F_j - Fv_j) (Eq. 1), formed
// from the contravariant velocity U_d = sum_j S[d][j] u_j: inviscid (rho U_d, rho u_i U_d +
// S[d][i] p, (E + p) U_d); viscous rows sigma_i = sum_j S[d][j] tau[i][j] and
// sum_i u_i sigma_i + sum_j S[d][j] hq[j].  Sd = S[d][0..2].
template <typename T>
__device__ __forceinline__ void contravariant_flux(const T q[5], const T u[3], T p, const T Sd[3], bool viscous,
                                                   const T tau[3][3], const T hq[3], T f[5]) {
  const T Ud = Sd[0] * u[0] + Sd[1] * u[1] + Sd[2] * u[2];
  f[0] = q[0] * Ud;
#pragma unroll
  for (int i = 0; i < 3; ++i) f[1 + i] = q[1 + i] * Ud + Sd[i] * p;
  f[4] = (q[4] + p) * Ud;
  if (viscous) {
    T sig[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      sig[i] = Sd[0] * tau[i][0] + Sd[1] * tau[i][1] + Sd[2] * tau[i][2];
      f[1 + i] = f[1 + i] - sig[i];
    }
    f[4] = f[4] - (u[0] * sig[0] + u[1] * sig[1] + u[2] * sig[2] + (Sd[0] * hq[0] + Sd[1] * hq[1] + Sd[2] * hq[2]));
  }
}

// ------------------------------------------------------------------------------------------
// Output or RK44 stage update of solution point t (flat point index over all elements): rv is the
// bracket of Eq. 3 at the point, s = -1/|J|.  MODE_RESIDUAL writes R; MODE_RK updates the FP64
// registers (acc, U_n) and the stage state (FP64 Q, or its double-float copy Qc on the mixed
// path) and ORs a non-finite result into *flag at the last stage.
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void finish_point(int64_t t, const T rv[5], T s, int mode, int stage, double dt,
                                             double *__restrict__ Rout, double *__restrict__ Q, T *__restrict__ Qc,
                                             double *__restrict__ Un, T *__restrict__ Unc, double *__restrict__ acc,
                                             int *__restrict__ flag, const DevPhys &dph) {
  double rd[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) rd[v] = to_double(rv[v] * s);
  if (dph.src_body || dph.src_sponge) {
    // Source term at the state the residual was evaluated on (the element kernels' input).
    double q[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v] = Qc ? to_double(Qc[t * 5 + v]) : Q[t * 5 + v];
    if (dph.src_body) {
      rd[1] += q[0] * dph.accel[0];
      rd[2] += q[0] * dph.accel[1];
      rd[3] += q[0] * dph.accel[2];
      rd[4] += q[1] * dph.accel[0] + q[2] * dph.accel[1] + q[3] * dph.accel[2];
    }
    if (dph.src_sponge) {
      const double sg = dph.sigma[t];
#pragma unroll
      for (int v = 0; v < 5; ++v) rd[v] -= sg * (q[v] - dph.Q_ref[t * 5 + v]);
    }
  }
  if (mode == MODE_RESIDUAL) {
#pragma unroll
    for (int v = 0; v < 5; ++v) Rout[t * 5 + v] = rd[v];
    return;
  }
  if (mode == MODE_SSP33 || mode == MODE_SSP104) {
    // FP64 registers on both paths: U_n (start of the step), Q (stage state) and, for the ten-stage
    // scheme, acc (its second register); the mixed path also refreshes the double-float copy Qc.
    //   SSP(3,3):  Q <- a_k U_n + b_k (Q + dt R), (a, b) = (0, 1), (3/4, 1/4), (1/3, 2/3).
    //   SSP(10,4): Q <- Q + dt/6 R at stages 0..8; after stage 4 the registers recombine,
    //              q2 = U_n/25 + 9/25 Q, Q <- 15 q2 - 5 Q; stage 9: Q <- q2 + 3/5 Q + dt/10 R.
    const int last = mode == MODE_SSP33 ? 2 : 9;
    bool bad = false;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const int64_t o = t * 5 + v;
      const double q = Q[o];
      double nq;
      if (mode == MODE_SSP33) {
        const double a = stage == 0 ? 0.0 : (stage == 1 ? 0.75 : 1.0 / 3.0);
        const double b = stage == 0 ? 1.0 : (stage == 1 ? 0.25 : 2.0 / 3.0);
        nq = a * Un[o] + b * fma(dt, rd[v], q);
      } else if (stage < 9) {
        nq = fma(dt / 6.0, rd[v], q);
        if (stage == 4) {
          const double q2 = Un[o] / 25.0 + 9.0 / 25.0 * nq;
          acc[o] = q2;
          nq = 15.0 * q2 - 5.0 * nq;
        }
      } else {
        nq = acc[o] + 0.6 * q + 0.1 * dt * rd[v];
      }
      Q[o] = nq;
      if constexpr (std::is_same<T, df32>::value) Qc[o] = from_double<T>(nq);
      if (stage == last) {
        Un[o] = nq;
        if constexpr (std::is_same<T, df32>::value) Unc[o] = from_double<T>(nq);
        bad |= !isfinite(nq);
      }
    }
    if (bad) atomicOr(flag, 1);
    return;
  }
  // RK44 weights b_k = (1/6, 1/3, 1/3, 1/6) and next-stage coefficients a = (1/2, 1/2, 1), picked
  // with selects (a runtime-indexed local array would live in local memory).
  const double bk = (stage == 0 || stage == 3) ? 1.0 / 6.0 : 1.0 / 3.0;
  const double ak = stage < 2 ? 0.5 : 1.0;
  bool bad = false;
  if constexpr (std::is_same<T, df32>::value) {
    // Mixed path: acc and U_n are FP64; the next stage state, read only by the element
    // kernels, is formed in double-float from the df32 copy of U_n.
    const T adt = from_double<T>(stage < 3 ? ak * dt : 0.0);
    if (stage < 3 && (dph.src_body || dph.src_sponge)) {
      // With a source term the stage increment comes from the FP64 residual, which includes S
      // (a separate uniform branch: the conversion costs FP64 work the plain path does without).
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const int64_t o = t * 5 + v;
        acc[o] = fma(bk * dt, rd[v], stage == 0 ? 0.0 : acc[o]);
        Qc[o] = Unc[o] + adt * from_double<T>(rd[v]);
      }
      return;
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const int64_t o = t * 5 + v;
      if (stage < 3) {
        acc[o] = fma(bk * dt, rd[v], stage == 0 ? 0.0 : acc[o]);
        Qc[o] = Unc[o] + adt * (rv[v] * s);
      } else {
        const double nv = fma(bk * dt, rd[v], Un[o] + acc[o]);
        Un[o] = nv;
        Q[o] = nv;
        const T nc = from_double<T>(nv);
        Unc[o] = nc;
        Qc[o] = nc;
        bad |= !isfinite(nv);
      }
    }
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const int64_t o = t * 5 + v;
      const double un = Un[o];
      if (stage < 3) {
        const double a_ = (stage == 0 ? 0.0 : acc[o]) + bk * dt * rd[v];
        acc[o] = a_;
        Q[o] = un + ak * dt * rd[v];
      } else {
        const double nv = un + acc[o] + bk * dt * rd[v];
        Un[o] = nv;
        Q[o] = nv;
        bad |= !isfinite(nv);
      }
    }
  }
  if (bad) atomicOr(flag, 1);
}

}  // namespace frx
