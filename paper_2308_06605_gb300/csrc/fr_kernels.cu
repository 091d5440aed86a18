// Per-mesh launches of the hexahedral FR kernels and their host-side dispatch (the device bodies
// are in fr_bodies.cuh); dt estimate; basis-table upload for every translation unit; dispatch of
// the batched stage kernel variants.
#include <algorithm>

#include "fr_bodies.cuh"

namespace frx {

// Copies of the FP64 state in the compute type (mixed path): the stage state and U_n.
__global__ void k_state_to_df(const double *__restrict__ Q, df32 *__restrict__ Qc, df32 *__restrict__ Unc,
                              int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) Qc[t] = Unc[t] = df_from(Q[t]);
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

template <int N, typename T>
static cudaError_t residual_impl(const DevMesh &m, const DevPhys &ph, int mode, int stage, double dt,
                                 double *Rout, cudaStream_t st, const PhaseEvents *ev, int phases) {
  constexpr int Np = N * N * N, Nf = N * N;
  const int64_t E = m.E;
  const T *Qin = reinterpret_cast<const T *>(m.mixed ? m.Qc : m.Q);
  T *Qtr = reinterpret_cast<T *>(m.Qtr), *Gtr = reinterpret_cast<T *>(m.Gtr), *FI = reinterpret_cast<T *>(m.FI);
  T *Rpart = reinterpret_cast<T *>(m.Rpart);
  const T *met = reinterpret_cast<const T *>(m.metrics), *lift = reinterpret_cast<const T *>(m.liftfac);
  const T *nrm = reinterpret_cast<const T *>(m.normals);
  T *Qc = m.mixed ? reinterpret_cast<T *>(m.Qc) : nullptr;
  const bool tri = m.if_tri != nullptr;
  cudaError_t err;
  if (phases & 1) {
    const int64_t n = E * 6 * Nf;
    FR_EV_BEGIN(0);
    // Double-float: staged through shared memory (measured 35 % faster at 48^3, p = 4); FP64: one
    // thread per face point reading the state directly (the staged form was 7 % slower there).
    if constexpr (std::is_same<T, df32>::value) {
      constexpr int epb = interp_epb<N>();
      if (n > 0 && m.tc) {
        if ((err = launch_interp_tc(m, st)) != cudaSuccess) return err;
      } else if (n > 0) {
        k_interp_faces_smem<N, T><<<(unsigned)((E + epb - 1) / epb), kInterpThreads, 0, st>>>(Qin, m.ef, Qtr, E);
      }
    } else if (n > 0) {
      k_interp_faces<N, T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Qin, m.ef, Qtr, E);
    }
    if ((err = launch_prism_phase(m, ph, 0, mode, stage, dt, Rout, st)) != cudaSuccess) return err;
    const int64_t nb = (m.n_if - m.n_interior) * Nf;
    if (nb > 0 && !tri)
      k_bc_prepare<N, T><<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(Qtr, nrm, m.if_bc, m.bcs, m.n_interior,
                                                                      m.n_if - m.n_interior, ph);
    if (nb > 0 && tri)
      k_bc_prepare_tri<N, T><<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(Qtr, nrm, m.if_bc, m.bcs, m.n_interior,
                                                                          m.n_if - m.n_interior, ph, m.if_tri);
    FR_EV_END(0);
  }
  if (phases & 2) {
    const int threads = volume_threads<N>();
    const size_t smem = sizeof(T) * (35 * Np + 30 * Nf) + (ph.closure ? sizeof(float) * (10 * Np + 1 + 128) : 0);
    // Double-float path with the viscous branch in FP32 (FR_PREC_MIXED_VF32), or the element
    // arithmetic throughout.
    auto kern = k_volume<N, T, false>;
    if constexpr (std::is_same<T, df32>::value)
      if (m.vf32) kern = k_volume<N, T, true>;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    FR_EV_BEGIN(1);
    if (E > 0 && ph.vc_basis) {
      if ((err = launch_vcjh_phase(m, ph, 1, mode, stage, dt, Rout, st)) != cudaSuccess) return err;
    } else if (E > 0) {
      kern<<<(unsigned)E, threads, smem, st>>>(Qin, met, m.ef, Qtr, lift, Gtr, Rpart, ph, m.h, m.nu, m.if_up,
                                               m.n_interior);
    }
    if ((err = launch_prism_phase(m, ph, 1, mode, stage, dt, Rout, st)) != cudaSuccess) return err;
    FR_EV_END(1);
  }
  if (phases & 4) {
    const int64_t n = m.n_interior * Nf;
    FR_EV_BEGIN(2);
    if (n > 0 && !tri) {
      auto ik = k_iface_flux<N, T, false>;
      if constexpr (std::is_same<T, df32>::value)
        if (m.vf32) ik = k_iface_flux<N, T, true>;
      ik<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(Qtr, Gtr, nrm, FI, m.n_interior, ph, m.if_elem, m.nu, m.if_up);
    }
    if (n > 0 && tri)
      k_iface_flux_tri<N, T><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(Qtr, Gtr, nrm, FI, m.n_interior, ph,
                                                                         m.if_elem, m.nu, m.if_tri, m.if_up);
    const int64_t nb = (m.n_if - m.n_interior) * Nf;
    if (nb > 0 && !tri)
      k_bc_flux<N, T><<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(Qtr, Gtr, nrm, m.if_bc, m.bcs, FI, m.n_interior,
                                                                   m.n_if - m.n_interior, ph, m.if_elem, m.nu);
    if (nb > 0 && tri)
      k_bc_flux_tri<N, T><<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(Qtr, Gtr, nrm, m.if_bc, m.bcs, FI,
                                                                       m.n_interior, m.n_if - m.n_interior, ph,
                                                                       m.if_elem, m.nu, m.if_tri);
    FR_EV_END(2);
  }
  if (phases & 8) {
    const int64_t n = E * Np;
    FR_EV_BEGIN(3);
    if (n > 0 && ph.vc_basis) {
      if ((err = launch_vcjh_phase(m, ph, 3, mode, stage, dt, Rout, st)) != cudaSuccess) return err;
    } else if (n > 0)
      k_correct<N, T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Rpart, FI, m.ef, met, E, mode, stage, dt, Rout,
                                                                   m.Q, Qc, m.Un, reinterpret_cast<T *>(m.Unc),
                                                                   m.acc, m.flag, ph);
    if ((err = launch_prism_phase(m, ph, 3, mode, stage, dt, Rout, st)) != cudaSuccess) return err;
    FR_EV_END(3);
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t dispatch_residual(const DevMesh &m, const DevPhys &ph, int mode, int stage, double dt,
                                     double *Rout, cudaStream_t st, const PhaseEvents *ev, int phases) {
  switch (m.N) {
    case 2: return residual_impl<2, T>(m, ph, mode, stage, dt, Rout, st, ev, phases);
    case 3: return residual_impl<3, T>(m, ph, mode, stage, dt, Rout, st, ev, phases);
    case 4: return residual_impl<4, T>(m, ph, mode, stage, dt, Rout, st, ev, phases);
    case 5: return residual_impl<5, T>(m, ph, mode, stage, dt, Rout, st, ev, phases);
    case 6: return residual_impl<6, T>(m, ph, mode, stage, dt, Rout, st, ev, phases);
    case 7: return residual_impl<7, T>(m, ph, mode, stage, dt, Rout, st, ev, phases);
    case 8: return residual_impl<8, T>(m, ph, mode, stage, dt, Rout, st, ev, phases);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_residual(const DevMesh &m, const DevPhys &ph, int mode, int stage, double dt, double *Rout,
                            cudaStream_t st, const PhaseEvents *ev, int phases) {
  if (m.mixed) return dispatch_residual<df32>(m, ph, mode, stage, dt, Rout, st, ev, phases);
  return dispatch_residual<double>(m, ph, mode, stage, dt, Rout, st, ev, phases);
}

cudaError_t launch_state_copy(const DevMesh &m, cudaStream_t st) {
  if (!m.mixed) return cudaSuccess;
  const int64_t n = (m.E * m.Np + m.Ep * m.Npp) * 5;
  k_state_to_df<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m.Q, reinterpret_cast<df32 *>(m.Qc),
                                                             reinterpret_cast<df32 *>(m.Unc), n);
  return cudaGetLastError();
}

template <int N>
static cudaError_t max_dt_impl(const DevMesh &m, const DevPhys &ph, double cfl, double *d_out, cudaStream_t st) {
  if (m.E > 0) k_elem_dt<N><<<(unsigned)((m.E + 127) / 128), 128, 0, st>>>(m.Q, m.h, m.E, ph.gamma, cfl, m.dtbuf);
  cudaError_t err = launch_prism_dt(m, ph, cfl, st);
  if (err != cudaSuccess) return err;
  k_min_reduce<<<1, 1024, 0, st>>>(m.dtbuf, m.E + m.Ep, d_out);
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

// Halo traces of a domain-decomposed mesh: entry k of the halo list is interface slot
// code[k] = 2 I + s (this part's side s).  Pack copies this part's slot into buf[k] (nv values
// of Nf points); unpack copies buf[k] into the other side's slot.  Values are moved as 8-byte
// words, so FP64 and double-float traces travel bit for bit.
__global__ void k_halo_copy(unsigned long long *__restrict__ X, unsigned long long *__restrict__ buf,
                            const int64_t *__restrict__ code, int64_t n_halo, int nvNf, int unpack) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_halo * nvNf) return;
  const int64_t k = t / nvNf;
  const int c = (int)(t - k * nvNf);
  const int64_t slot = unpack ? (code[k] ^ 1) : code[k];
  if (unpack)
    X[slot * nvNf + c] = buf[t];
  else
    buf[t] = X[slot * nvNf + c];
}

cudaError_t launch_halo_copy(double *X, double *buf, const int64_t *code, int64_t n_halo, int nv, int Nf, int unpack,
                             cudaStream_t st) {
  const int64_t n = n_halo * nv * Nf;
  if (n == 0) return cudaSuccess;
  k_halo_copy<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<unsigned long long *>(X),
                                                           reinterpret_cast<unsigned long long *>(buf), code, n_halo,
                                                           nv * Nf, unpack);
  return cudaGetLastError();
}

// OR the per-case non-finite flags into the batch word and clear them (graph-of-kernels mode).
__global__ void k_gather_flags(const BatchCase *cases, int n, BatchSync *sy) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int *f = cases[i].m.flag;
    if (*f) {
      atomicOr(&sy->nonfinite, 1);
      *f = 0;
    }
  }
}

cudaError_t launch_gather_flags(const BatchCase *cases, int n, BatchSync *sy, cudaStream_t st) {
  k_gather_flags<<<1, 128, 0, st>>>(cases, n, sy);
  return cudaGetLastError();
}

size_t batch_smem_bytes(const int *Ns, const int *has_prism, int n, int block, int mixed) {
  (void)mixed;
  size_t best = 0;
  for (int k = 0; k < n; ++k) {
    const int N = Ns[k];
    const size_t hex = (size_t)(35 * N * N * N + 30 * N * N) * sizeof(double) * batch_elems_per_block(N, block);
    best = std::max(best, hex);
    if (has_prism[k]) {
      const size_t per = (size_t)(65 * (N * (N + 1) / 2 * N) + 25 * N * N) * sizeof(double);
      best = std::max(best, per * batch_prism_elems_per_block(N, block));
    }
  }
  return best;
}

cudaError_t upload_basis_tables() {
  cudaError_t e = upload_basis_local();
  if (e == cudaSuccess) e = upload_tc_tables();
  if (e == cudaSuccess) e = batch_upload_m0_b256();
  if (e == cudaSuccess) e = batch_upload_m0_b512();
  if (e == cudaSuccess) e = batch_upload_m1_b256();
  if (e == cudaSuccess) e = batch_upload_m1_b512();
  return e;
}

cudaError_t launch_batch_stage(const BatchLaunch &L, int mixed, int block, int grid, size_t smem, cudaStream_t st) {
  if (block == 256) return mixed ? batch_launch_m1_b256(L, grid, smem, st) : batch_launch_m0_b256(L, grid, smem, st);
  if (block == 512) return mixed ? batch_launch_m1_b512(L, grid, smem, st) : batch_launch_m0_b512(L, grid, smem, st);
  return cudaErrorInvalidValue;
}

cudaError_t batch_occupancy(int mixed, int block, size_t smem, int *nb) {
  if (block == 256) return mixed ? batch_occupancy_m1_b256(smem, nb) : batch_occupancy_m0_b256(smem, nb);
  if (block == 512) return mixed ? batch_occupancy_m1_b512(smem, nb) : batch_occupancy_m0_b512(smem, nb);
  return cudaErrorInvalidValue;
}

}  // namespace frx
