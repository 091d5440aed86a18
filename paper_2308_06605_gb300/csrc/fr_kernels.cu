// FP64 kernels of the FR residual and the RK44 stage update (arXiv 2308.06605, section
// "FR Algorithm", Eq. 1-3).  One residual evaluation is four launches:
//   interp_faces : Q -> solution traces at the flux points of every face (interface slots)
//   volume       : per element, BR2-corrected gradients, physical + transformed fluxes at the
//                  solution points, gradient traces at the flux points, and the divergence of
//                  the transformed flux including the own-flux part of the correction
//   iface_flux   : per interface flux point, Rusanov + BR2 common normal flux
//   correct      : per solution point, adds the common-flux correction, scales by -1/|J| and
//                  writes R or applies the RK44 stage update.
#include <cuda_runtime.h>

#include <cmath>

#include "fr_device.hpp"

namespace frx {

__constant__ DevBasis c_basis[kMaxN];   // index N - 1 (N = 2..8 used)

cudaError_t upload_basis_tables() {
  DevBasis hb[kMaxN] = {};
  for (int p = 1; p < kMaxN; ++p) {
    Basis1D b = make_basis(p);
    const int N = p + 1;
    DevBasis &d = hb[N - 1];
    for (int i = 0; i < N; ++i) {
      d.lm[i] = b.lm[i];
      d.lp[i] = b.lp[i];
      d.hm[i] = b.hm[i];
      d.hp[i] = b.hp[i];
      for (int a = 0; a < N; ++a) {
        d.D[i * N + a] = b.D[i * N + a];
        d.Dt[i * N + a] = b.D[i * N + a] - b.hp[i] * b.lp[a] + b.hm[i] * b.lm[a];
      }
    }
  }
  return cudaMemcpyToSymbol(c_basis, hb, sizeof(hb));
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

// ------------------------------------------------------------------------------------------
// Gas dynamics (ideal gas, Stokes hypothesis, constant mu, Fourier heat flux).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void normal_inviscid(const double q[5], const double n[3], double g,
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
  const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  un_abs_plus_c_n = fabs(un) + sqrt(g * p * ri) * nn;      // (|u.n^| + c) |n|
}

// Viscous flux F_v[j][v] (j = direction) of state q with gradient G[j*5 + v] = dQ_v/dx_j.
__device__ __forceinline__ void viscous_flux(const double q[5], const double *G, const DevPhys &ph,
                                             double Fv[3][5]) {
  const double ri = 1.0 / q[0];
  const double u[3] = {q[1] * ri, q[2] * ri, q[3] * ri};
  const double eo = q[4] * ri;
  double du[3][3];   // du[i][j] = du_i/dx_j
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) du[i][j] = (G[j * 5 + 1 + i] - u[i] * G[j * 5]) * ri;
  double dT[3];
  const double cT = (ph.gamma - 1.0) / ph.R;
#pragma unroll
  for (int j = 0; j < 3; ++j)
    dT[j] = cT * ((G[j * 5 + 4] - eo * G[j * 5]) * ri - (u[0] * du[0][j] + u[1] * du[1][j] + u[2] * du[2][j]));
  const double lam = -2.0 / 3.0 * ph.mu * (du[0][0] + du[1][1] + du[2][2]);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    double t[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) t[i] = ph.mu * (du[i][j] + du[j][i]) + (i == j ? lam : 0.0);
    Fv[j][0] = 0.0;
    Fv[j][1] = t[0];
    Fv[j][2] = t[1];
    Fv[j][3] = t[2];
    Fv[j][4] = u[0] * t[0] + u[1] * t[1] + u[2] * t[2] + ph.kappa * dT[j];
  }
}

// ------------------------------------------------------------------------------------------
// 1. Solution traces.  Thread per (element, face, flux point).
// ------------------------------------------------------------------------------------------
template <int N>
__global__ void k_interp_faces(const double *__restrict__ Q, const int32_t *__restrict__ ef,
                               double *__restrict__ Qtr, int64_t E) {
  constexpr int Np = N * N * N, Nf = N * N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= E * 6 * Nf) return;
  const int r = (int)(t % Nf);
  const int64_t eff = t / Nf;
  const int f = (int)(eff % 6);
  const int64_t e = eff / 6;
  const DevBasis &B = c_basis[N - 1];
  const double *l = (f & 1) ? B.lp : B.lm;
  int base, sd;
  face_line<N>(f, r, base, sd);
  const double *q = Q + e * Np * 5;
  double acc[5] = {0, 0, 0, 0, 0};
#pragma unroll
  for (int c = 0; c < N; ++c) {
    const double lc = l[c];
    const double *qc = q + (base + c * sd) * 5;
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += lc * qc[v];
  }
  const int packed = ef[eff];
  const int64_t I = packed >> 4;
  const int side = (packed >> 3) & 1;
  const int slot = slot_of(packed & 7, r % N, r / N, N);
  double *dst = Qtr + (I * 2 + side) * 5 * Nf + slot;
#pragma unroll
  for (int v = 0; v < 5; ++v) dst[v * Nf] = acc[v];
}

// ------------------------------------------------------------------------------------------
// 2. Volume kernel.  One block per element, one thread per solution point.
// ------------------------------------------------------------------------------------------
template <int N>
__global__ void k_volume(const double *__restrict__ Q, const double *__restrict__ metrics,
                         const int32_t *__restrict__ ef, const double *__restrict__ Qtr,
                         const double *__restrict__ liftfac, double *__restrict__ Gtr,
                         double *__restrict__ Rpart, DevPhys ph) {
  constexpr int Np = N * N * N, Nf = N * N;
  extern __shared__ double sm[];
  double *sQ = sm;                 // [5][Np]
  double *sG = sQ + 5 * Np;        // [15][Np] uncorrected physical gradient, index j*5+v
  double *sH = sG + 15 * Np;       // [15][Np] transformed flux, index d*5+v
  double *sdQ = sH + 15 * Np;      // [6][5][Nf] Q^I - Q_own at the flux points
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x;
  const DevBasis &B = c_basis[N - 1];
  const bool viscous = ph.viscous != 0;
  for (int t = tid; t < 5 * Np; t += blockDim.x) sQ[(t % 5) * Np + t / 5] = Q[e * Np * 5 + t];
  if (viscous) {
    for (int t = tid; t < 6 * Nf; t += blockDim.x) {
      const int f = t / Nf, r = t % Nf;
      const int packed = ef[e * 6 + f];
      const int64_t I = packed >> 4;
      const int side = (packed >> 3) & 1;
      const int slot = slot_of(packed & 7, r % N, r / N, N);
      const double *own = Qtr + (I * 2 + side) * 5 * Nf + slot;
      const double *oth = Qtr + (I * 2 + (1 - side)) * 5 * Nf + slot;
#pragma unroll
      for (int v = 0; v < 5; ++v) sdQ[(f * 5 + v) * Nf + r] = 0.5 * (oth[v * Nf] - own[v * Nf]);
    }
  }
  __syncthreads();
  if (tid < Np) {
    const int m = tid, i = m % N, j = (m / N) % N, k = m / (N * N);
    double S[9];
    const double *met = metrics + e * 10 * Np + m;
#pragma unroll
    for (int c = 0; c < 9; ++c) S[c] = met[c * Np];
    const double invJ = met[9 * Np];
    double q[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v] = sQ[v * Np + m];
    double H[3][5];
    {
      // Inviscid flux F_j.
      const double ri = 1.0 / q[0];
      const double u[3] = {q[1] * ri, q[2] * ri, q[3] * ri};
      const double p = (ph.gamma - 1.0) * (q[4] - 0.5 * (q[1] * u[0] + q[2] * u[1] + q[3] * u[2]));
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) {
        H[jj][0] = q[1 + jj];
        H[jj][1] = q[1] * u[jj] + (jj == 0 ? p : 0.0);
        H[jj][2] = q[2] * u[jj] + (jj == 1 ? p : 0.0);
        H[jj][3] = q[3] * u[jj] + (jj == 2 ? p : 0.0);
        H[jj][4] = (q[4] + p) * u[jj];
      }
    }
    if (viscous) {
      double gu[3][5], gc[3][5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double *sq = sQ + v * Np;
        double a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
        for (int a = 0; a < N; ++a) {
          a0 += B.D[i * N + a] * sq[a + N * j + N * N * k];
          a1 += B.D[j * N + a] * sq[i + N * a + N * N * k];
          a2 += B.D[k * N + a] * sq[i + N * j + N * N * a];
        }
        gu[0][v] = a0;
        gu[1][v] = a1;
        gu[2][v] = a2;
        gc[0][v] = a0 - B.hm[i] * sdQ[(0 * 5 + v) * Nf + j + N * k] + B.hp[i] * sdQ[(1 * 5 + v) * Nf + j + N * k];
        gc[1][v] = a1 - B.hm[j] * sdQ[(2 * 5 + v) * Nf + i + N * k] + B.hp[j] * sdQ[(3 * 5 + v) * Nf + i + N * k];
        gc[2][v] = a2 - B.hm[k] * sdQ[(4 * 5 + v) * Nf + i + N * j] + B.hp[k] * sdQ[(5 * 5 + v) * Nf + i + N * j];
      }
      double G[15];
#pragma unroll
      for (int jj = 0; jj < 3; ++jj)
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const double s0 = S[0 * 3 + jj] * invJ, s1 = S[1 * 3 + jj] * invJ, s2 = S[2 * 3 + jj] * invJ;
          sG[(jj * 5 + v) * Np + m] = s0 * gu[0][v] + s1 * gu[1][v] + s2 * gu[2][v];
          G[jj * 5 + v] = s0 * gc[0][v] + s1 * gc[1][v] + s2 * gc[2][v];
        }
      double Fv[3][5];
      viscous_flux(q, G, ph, Fv);
#pragma unroll
      for (int jj = 0; jj < 3; ++jj)
#pragma unroll
        for (int v = 0; v < 5; ++v) H[jj][v] -= Fv[jj][v];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int v = 0; v < 5; ++v)
        sH[(d * 5 + v) * Np + m] = S[d * 3 + 0] * H[0][v] + S[d * 3 + 1] * H[1][v] + S[d * 3 + 2] * H[2][v];
  }
  __syncthreads();
  if (viscous) {
    // Gradient traces: uncorrected gradient interpolated to the face + eta * own lifting.
    for (int t = tid; t < 6 * Nf; t += blockDim.x) {
      const int f = t / Nf, r = t % Nf;
      const double *l = (f & 1) ? B.lp : B.lm;
      int base, sd;
      face_line<N>(f, r, base, sd);
      const int packed = ef[e * 6 + f];
      const int64_t I = packed >> 4;
      const int side = (packed >> 3) & 1;
      const int slot = slot_of(packed & 7, r % N, r / N, N);
      double *dst = Gtr + (I * 2 + side) * 15 * Nf + slot;
      const double *lf = liftfac + (e * 6 + f) * 3 * Nf + r;
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) {
        const double lj = ph.eta * lf[jj * Nf];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const double *sg = sG + (jj * 5 + v) * Np + base;
          double acc = 0.0;
#pragma unroll
          for (int c = 0; c < N; ++c) acc += l[c] * sg[c * sd];
          dst[(jj * 5 + v) * Nf] = acc + lj * sdQ[(f * 5 + v) * Nf + r];
        }
      }
    }
  }
  if (tid < Np) {
    const int m = tid, i = m % N, j = (m / N) % N, k = m / (N * N);
    double *out = Rpart + (e * Np + m) * 5;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double *h0 = sH + (0 * 5 + v) * Np, *h1 = sH + (1 * 5 + v) * Np, *h2 = sH + (2 * 5 + v) * Np;
      double acc = 0.0;
#pragma unroll
      for (int a = 0; a < N; ++a) {
        acc += B.Dt[i * N + a] * h0[a + N * j + N * N * k];
        acc += B.Dt[j * N + a] * h1[i + N * a + N * N * k];
        acc += B.Dt[k * N + a] * h2[i + N * j + N * N * a];
      }
      out[v] = acc;
    }
  }
}

// ------------------------------------------------------------------------------------------
// 3. Common normal flux at the flux points of two-sided interfaces (Rusanov + BR2).
// ------------------------------------------------------------------------------------------
template <int N>
__global__ void k_iface_flux(const double *__restrict__ Qtr, const double *__restrict__ Gtr,
                             const double *__restrict__ normals, double *__restrict__ FI,
                             int64_t n_if, DevPhys ph) {
  constexpr int Nf = N * N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_if * Nf) return;
  const int64_t I = t / Nf;
  const int q = (int)(t % Nf);
  double qL[5], qR[5], n[3];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qL[v] = Qtr[(I * 2 + 0) * 5 * Nf + v * Nf + q];
    qR[v] = Qtr[(I * 2 + 1) * 5 * Nf + v * Nf + q];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) n[c] = normals[(I * 3 + c) * Nf + q];
  double fL[5], fR[5], sL, sR;
  normal_inviscid(qL, n, ph.gamma, fL, sL);
  normal_inviscid(qR, n, ph.gamma, fR, sR);
  const double lam = fmax(sL, sR);
  double F[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * lam * (qR[v] - qL[v]);
  if (ph.viscous) {
    double qc[5], G[15];
#pragma unroll
    for (int v = 0; v < 5; ++v) qc[v] = 0.5 * (qL[v] + qR[v]);
#pragma unroll
    for (int c = 0; c < 15; ++c)
      G[c] = 0.5 * (Gtr[(I * 2 + 0) * 15 * Nf + c * Nf + q] + Gtr[(I * 2 + 1) * 15 * Nf + c * Nf + q]);
    double Fv[3][5];
    viscous_flux(qc, G, ph, Fv);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] -= Fv[0][v] * n[0] + Fv[1][v] * n[1] + Fv[2][v] * n[2];
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) FI[(I * 5 + v) * Nf + q] = F[v];
}

// ------------------------------------------------------------------------------------------
// 3b. Boundary faces.  Side 0 of a boundary interface is the element; its side-1 slot holds
// 2 Q^I - Q- so that the volume kernel's (other - own)/2 equals Q^I - Q- for the BR2 jump.
// ------------------------------------------------------------------------------------------
// Ghost state (for the Rusanov flux) and boundary common solution Q^I from the interior trace.
__device__ void boundary_states(const double qm[5], const double n[3], const fr_bc &bc, const DevPhys &ph,
                                double ghost[5], double qi[5]) {
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
  const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
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

template <int N>
__global__ void k_bc_prepare(double *__restrict__ Qtr, const double *__restrict__ normals,
                             const int32_t *__restrict__ if_bc, const fr_bc *__restrict__ bcs,
                             int64_t first, int64_t count, DevPhys ph) {
  constexpr int Nf = N * N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count * Nf) return;
  const int64_t I = first + t / Nf;
  const int q = (int)(t % Nf);
  double qm[5], n[3], gh[5], qi[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) qm[v] = Qtr[(I * 2 + 0) * 5 * Nf + v * Nf + q];
#pragma unroll
  for (int c = 0; c < 3; ++c) n[c] = normals[(I * 3 + c) * Nf + q];
  boundary_states(qm, n, bcs[if_bc[I]], ph, gh, qi);
#pragma unroll
  for (int v = 0; v < 5; ++v) Qtr[(I * 2 + 1) * 5 * Nf + v * Nf + q] = 2.0 * qi[v] - qm[v];
}

template <int N>
__global__ void k_bc_flux(const double *__restrict__ Qtr, const double *__restrict__ Gtr,
                          const double *__restrict__ normals, const int32_t *__restrict__ if_bc,
                          const fr_bc *__restrict__ bcs, double *__restrict__ FI, int64_t first,
                          int64_t count, DevPhys ph) {
  constexpr int Nf = N * N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count * Nf) return;
  const int64_t I = first + t / Nf;
  const int q = (int)(t % Nf);
  double qm[5], n[3], gh[5], qi[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) qm[v] = Qtr[(I * 2 + 0) * 5 * Nf + v * Nf + q];
#pragma unroll
  for (int c = 0; c < 3; ++c) n[c] = normals[(I * 3 + c) * Nf + q];
  boundary_states(qm, n, bcs[if_bc[I]], ph, gh, qi);
  double fL[5], fR[5], sL, sR;
  normal_inviscid(qm, n, ph.gamma, fL, sL);
  normal_inviscid(gh, n, ph.gamma, fR, sR);
  const double lam = fmax(sL, sR);
  double F[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * lam * (gh[v] - qm[v]);
  if (ph.viscous) {
    double G[15];
#pragma unroll
    for (int c = 0; c < 15; ++c) G[c] = Gtr[(I * 2 + 0) * 15 * Nf + c * Nf + q];
    double Fv[3][5];
    viscous_flux(qi, G, ph, Fv);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] -= Fv[0][v] * n[0] + Fv[1][v] * n[1] + Fv[2][v] * n[2];
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) FI[(I * 5 + v) * Nf + q] = F[v];
}

// ------------------------------------------------------------------------------------------
// 4. Correction by the common flux, scaling, and output / RK44 stage update.
// ------------------------------------------------------------------------------------------
template <int N>
__global__ void k_correct(const double *__restrict__ Rpart, const double *__restrict__ FI,
                          const int32_t *__restrict__ ef, const double *__restrict__ metrics,
                          int64_t E, int mode, int stage, double dt, double *__restrict__ Rout,
                          double *__restrict__ Q, double *__restrict__ Un, double *__restrict__ acc,
                          int *__restrict__ flag) {
  constexpr int Np = N * N * N, Nf = N * N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= E * Np) return;
  const int64_t e = t / Np;
  const int m = (int)(t % Np), i = m % N, j = (m / N) % N, k = m / (N * N);
  const DevBasis &B = c_basis[N - 1];
  double r[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) r[v] = Rpart[t * 5 + v];
  // Faces: (f, weight, local flux point (a, b)).
  const int fa[6] = {j, j, i, i, i, i};
  const int fb[6] = {k, k, k, k, j, j};
  const double wts[6] = {B.hm[i], B.hp[i], B.hm[j], B.hp[j], B.hm[k], B.hp[k]};
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int packed = ef[e * 6 + f];
    const int64_t I = packed >> 4;
    const int side = (packed >> 3) & 1;
    const int slot = slot_of(packed & 7, fa[f], fb[f], N);
    const double w = side ? -wts[f] : wts[f];
    const double *src = FI + I * 5 * Nf + slot;
#pragma unroll
    for (int v = 0; v < 5; ++v) r[v] += w * src[v * Nf];
  }
  const double s = -metrics[(e * 10 + 9) * Np + m];
#pragma unroll
  for (int v = 0; v < 5; ++v) r[v] *= s;
  if (mode == MODE_RESIDUAL) {
#pragma unroll
    for (int v = 0; v < 5; ++v) Rout[t * 5 + v] = r[v];
    return;
  }
  const double bcoef[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  const double anext[3] = {0.5, 0.5, 1.0};
  bool bad = false;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const int64_t o = t * 5 + v;
    const double un = Un[o];
    if (stage < 3) {
      const double a_ = (stage == 0 ? 0.0 : acc[o]) + bcoef[stage] * dt * r[v];
      acc[o] = a_;
      Q[o] = un + anext[stage] * dt * r[v];
    } else {
      const double nv = un + acc[o] + bcoef[3] * dt * r[v];
      Un[o] = nv;
      Q[o] = nv;
      bad |= !isfinite(nv);
    }
  }
  if (bad) atomicOr(flag, 1);
}

// ------------------------------------------------------------------------------------------
// dt estimate: per element max(|u| + c) -> h / ((2p+1) lambda); then a block-level min.
// ------------------------------------------------------------------------------------------
template <int N>
__global__ void k_elem_dt(const double *__restrict__ Q, const double *__restrict__ h, int64_t E,
                          double gamma, double cfl, double *__restrict__ dte) {
  constexpr int Np = N * N * N;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  double lam = 0.0;
  for (int m = 0; m < Np; ++m) {
    const double *q = Q + (e * Np + m) * 5;
    const double ri = 1.0 / q[0];
    const double u = q[1] * ri, v = q[2] * ri, w = q[3] * ri;
    const double p = (gamma - 1.0) * (q[4] - 0.5 * (q[1] * u + q[2] * v + q[3] * w));
    lam = fmax(lam, sqrt(u * u + v * v + w * w) + sqrt(gamma * p * ri));
  }
  dte[e] = cfl * h[e] / ((2 * (N - 1) + 1) * lam);
}

__global__ void k_min_reduce(const double *__restrict__ x, int64_t n, double *__restrict__ out) {
  __shared__ double s[1024];
  double v = INFINITY;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v = fmin(v, x[i]);
  s[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] = fmin(s[threadIdx.x], s[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// ------------------------------------------------------------------------------------------
#define FR_EV_BEGIN(k) \
  if (ev) cudaEventRecord(ev->start[k], st)
#define FR_EV_END(k) \
  if (ev) cudaEventRecord(ev->stop[k], st)

template <int N>
static cudaError_t residual_impl(const DevMesh &m, const DevPhys &ph, int mode, int stage, double dt,
                                 double *Rout, cudaStream_t st, const PhaseEvents *ev) {
  constexpr int Np = N * N * N, Nf = N * N;
  const int64_t E = m.E;
  {
    const int64_t n = E * 6 * Nf;
    FR_EV_BEGIN(0);
    k_interp_faces<N><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m.Q, m.ef, m.Qtr, E);
    const int64_t nb = (m.n_if - m.n_interior) * Nf;
    if (nb > 0)
      k_bc_prepare<N><<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(m.Qtr, m.normals, m.if_bc, m.bcs, m.n_interior,
                                                                   m.n_if - m.n_interior, ph);
    FR_EV_END(0);
  }
  {
    const int threads = ((Np + 31) / 32) * 32;
    const size_t smem = sizeof(double) * (35 * Np + 30 * Nf);
    static bool attr_set = false;
    if (!attr_set) {
      cudaError_t err = cudaFuncSetAttribute(k_volume<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
      attr_set = true;
    }
    FR_EV_BEGIN(1);
    k_volume<N><<<(unsigned)E, threads, smem, st>>>(m.Q, m.metrics, m.ef, m.Qtr, m.liftfac, m.Gtr, m.Rpart, ph);
    FR_EV_END(1);
  }
  {
    const int64_t n = m.n_interior * Nf;
    FR_EV_BEGIN(2);
    if (n > 0) k_iface_flux<N><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(m.Qtr, m.Gtr, m.normals, m.FI, m.n_interior, ph);
    const int64_t nb = (m.n_if - m.n_interior) * Nf;
    if (nb > 0)
      k_bc_flux<N><<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(m.Qtr, m.Gtr, m.normals, m.if_bc, m.bcs, m.FI,
                                                                m.n_interior, m.n_if - m.n_interior, ph);
    FR_EV_END(2);
  }
  {
    const int64_t n = E * Np;
    FR_EV_BEGIN(3);
    k_correct<N><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m.Rpart, m.FI, m.ef, m.metrics, E, mode, stage, dt,
                                                              Rout, m.Q, m.Un, m.acc, m.flag);
    FR_EV_END(3);
  }
  return cudaGetLastError();
}

cudaError_t launch_residual(const DevMesh &m, const DevPhys &ph, int mode, int stage, double dt, double *Rout,
                            cudaStream_t st, const PhaseEvents *ev) {
  switch (m.N) {
    case 2: return residual_impl<2>(m, ph, mode, stage, dt, Rout, st, ev);
    case 3: return residual_impl<3>(m, ph, mode, stage, dt, Rout, st, ev);
    case 4: return residual_impl<4>(m, ph, mode, stage, dt, Rout, st, ev);
    case 5: return residual_impl<5>(m, ph, mode, stage, dt, Rout, st, ev);
    case 6: return residual_impl<6>(m, ph, mode, stage, dt, Rout, st, ev);
    case 7: return residual_impl<7>(m, ph, mode, stage, dt, Rout, st, ev);
    case 8: return residual_impl<8>(m, ph, mode, stage, dt, Rout, st, ev);
    default: return cudaErrorInvalidValue;
  }
}

template <int N>
static cudaError_t max_dt_impl(const DevMesh &m, const DevPhys &ph, double cfl, double *d_out, cudaStream_t st) {
  k_elem_dt<N><<<(unsigned)((m.E + 127) / 128), 128, 0, st>>>(m.Q, m.h, m.E, ph.gamma, cfl, m.dtbuf);
  k_min_reduce<<<1, 1024, 0, st>>>(m.dtbuf, m.E, d_out);
  return cudaGetLastError();
}

cudaError_t launch_max_dt(const DevMesh &m, const DevPhys &ph, double cfl, double *d_out, cudaStream_t st) {
  switch (m.N) {
    case 2: return max_dt_impl<2>(m, ph, cfl, d_out, st);
    case 3: return max_dt_impl<3>(m, ph, cfl, d_out, st);
    case 4: return max_dt_impl<4>(m, ph, cfl, d_out, st);
    case 5: return max_dt_impl<5>(m, ph, cfl, d_out, st);
    case 6: return max_dt_impl<6>(m, ph, cfl, d_out, st);
    case 7: return max_dt_impl<7>(m, ph, cfl, d_out, st);
    case 8: return max_dt_impl<8>(m, ph, cfl, d_out, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace frx
