// Kernels of the FR residual on the prisms of mixed hexahedral/prismatic meshes (arXiv 2308.06605,
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
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "df32.cuh"
#include "fr_device.hpp"
#include "fr_point.cuh"
#include "fr_prism_bodies.cuh"

namespace frx {

// ------------------------------------------------------------------------------------------
// Per-mesh kernels: one launch per phase over all prisms of a mesh.
// ------------------------------------------------------------------------------------------
template <int N, typename T>
__global__ void k_prism_interp(const T *__restrict__ Q, const int32_t *__restrict__ ef_p, const T *__restrict__ tab,
                               const int32_t *__restrict__ tri_slot, T *__restrict__ Qtr, int64_t Ep) {
  prism_interp_body<N, T>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, Q, ef_p, tab, tri_slot, Qtr, Ep);
}

template <int N, typename T>
__global__ void __launch_bounds__(prism_threads<N>(), prism_min_blocks<N, T>())
    k_prism_volume(const T *__restrict__ Q, const T *__restrict__ metrics, const int32_t *__restrict__ ef_p,
                   const T *__restrict__ Qtr, const T *__restrict__ tab, const int32_t *__restrict__ tri_slot,
                   T *__restrict__ Gtr, T *__restrict__ Rpart, DevPhys dph, const int8_t *__restrict__ if_up,
                   int64_t n_interior) {
  extern __shared__ double sm_raw[];
  prism_volume_body<N, T>(blockIdx.x, threadIdx.x, blockDim.x, true, sm_raw, Q, metrics, ef_p, Qtr, tab, tri_slot,
                          Gtr, Rpart, dph, if_up, n_interior);
}

template <int N, typename T>
__global__ void k_prism_correct(const T *__restrict__ Rpart, const T *__restrict__ FI, const int32_t *__restrict__ ef_p,
                                const T *__restrict__ metrics, const T *__restrict__ tab,
                                const int32_t *__restrict__ tri_slot, int64_t Ep, int64_t first_point, int mode,
                                int stage, double dt, double *__restrict__ Rout, double *__restrict__ Q,
                                T *__restrict__ Qc, double *__restrict__ Un, T *__restrict__ Unc,
                                double *__restrict__ acc, int *__restrict__ flag, DevPhys dph) {
  prism_correct_body<N, T>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, Rpart, FI, ef_p, metrics, tab, tri_slot, Ep,
                           first_point, mode, stage, dt, Rout, Q, Qc, Un, Unc, acc, flag, dph);
}

// dt bound per prism: cfl h / ((2p + 1) max(|u| + c)) over its points (FP64 state).
__global__ void k_prism_dt(const double *__restrict__ Q, const double *__restrict__ h, int64_t Ep, int Npp, int p,
                           double gamma, double cfl, double *__restrict__ dte) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Ep) return;
  double lam = 0.0;
  for (int m = 0; m < Npp; ++m) {
    const double *q = Q + (e * Npp + m) * 5;
    const double ri = 1.0 / q[0];
    const double u = q[1] * ri, v = q[2] * ri, w = q[3] * ri;
    const double pr = (gamma - 1.0) * (q[4] - 0.5 * (q[1] * u + q[2] * v + q[3] * w));
    lam = fmax(lam, sqrt(u * u + v * v + w * w) + sqrt(gamma * pr * ri));
  }
  dte[e] = cfl * h[e] / ((2 * p + 1) * lam);
}

// ------------------------------------------------------------------------------------------
template <int N, typename T>
static cudaError_t prism_phase_impl(const DevMesh &m, const DevPhys &ph, int phase, int mode, int stage, double dt,
                                    double *Rout, cudaStream_t st) {
  constexpr int Nt = N * (N + 1) / 2, Np = Nt * N, Nf = N * N;
  if (m.Ep == 0) return cudaSuccess;
  if (m.Nt != Nt || m.Npp != Np) return cudaErrorInvalidValue;
  const int64_t off = m.E * m.Np * 5;                        // first prism value in per-point arrays
  const T *Qin = reinterpret_cast<const T *>(m.mixed ? m.Qc : m.Q) + off;
  const T *tab = reinterpret_cast<const T *>(m.ptab);
  const T *met = reinterpret_cast<const T *>(m.metrics_p);
  T *Qtr = reinterpret_cast<T *>(m.Qtr), *Gtr = reinterpret_cast<T *>(m.Gtr), *FI = reinterpret_cast<T *>(m.FI);
  T *Rpart = reinterpret_cast<T *>(m.Rpart) + off;
  if (phase == 0) {
    const int64_t n = m.Ep * 5 * Nf;
    k_prism_interp<N, T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Qin, m.ef_p, tab, m.tri_slot, Qtr, m.Ep);
  } else if (phase == 1) {
    const size_t smem = sizeof(T) * prism_smem_values<N>();
    cudaError_t err = cudaFuncSetAttribute(k_prism_volume<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_prism_volume<N, T><<<(unsigned)m.Ep, prism_threads<N>(), smem, st>>>(Qin, met, m.ef_p, Qtr, tab, m.tri_slot,
                                                                          Gtr, Rpart, ph, m.if_up, m.n_interior);
  } else if (phase == 3) {
    const int64_t n = m.Ep * Np;
    k_prism_correct<N, T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        Rpart, FI, m.ef_p, met, tab, m.tri_slot, m.Ep, m.E * m.Np, mode, stage, dt, Rout, m.Q,
        m.mixed ? reinterpret_cast<T *>(m.Qc) : nullptr, m.Un, reinterpret_cast<T *>(m.Unc), m.acc, m.flag, ph);
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t prism_dispatch(const DevMesh &m, const DevPhys &ph, int phase, int mode, int stage, double dt,
                                  double *Rout, cudaStream_t st) {
  switch (m.N) {
    case 2: return prism_phase_impl<2, T>(m, ph, phase, mode, stage, dt, Rout, st);
    case 3: return prism_phase_impl<3, T>(m, ph, phase, mode, stage, dt, Rout, st);
    case 4: return prism_phase_impl<4, T>(m, ph, phase, mode, stage, dt, Rout, st);
    case 5: return prism_phase_impl<5, T>(m, ph, phase, mode, stage, dt, Rout, st);
    case 6: return prism_phase_impl<6, T>(m, ph, phase, mode, stage, dt, Rout, st);
    case 7: return prism_phase_impl<7, T>(m, ph, phase, mode, stage, dt, Rout, st);
    case 8: return prism_phase_impl<8, T>(m, ph, phase, mode, stage, dt, Rout, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_prism_phase(const DevMesh &m, const DevPhys &ph, int phase, int mode, int stage, double dt,
                               double *Rout, cudaStream_t st) {
  if (m.Ep == 0) return cudaSuccess;
  if (m.mixed) return prism_dispatch<df32>(m, ph, phase, mode, stage, dt, Rout, st);
  return prism_dispatch<double>(m, ph, phase, mode, stage, dt, Rout, st);
}

cudaError_t launch_prism_dt(const DevMesh &m, const DevPhys &ph, double cfl, cudaStream_t st) {
  if (m.Ep == 0) return cudaSuccess;
  k_prism_dt<<<(unsigned)((m.Ep + 127) / 128), 128, 0, st>>>(m.Q + m.E * m.Np * 5, m.h + m.E, m.Ep, m.Npp, m.p,
                                                              ph.gamma, cfl, m.dtbuf + m.E);
  return cudaGetLastError();
}

}  // namespace frx
