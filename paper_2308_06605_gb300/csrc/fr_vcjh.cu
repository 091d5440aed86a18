// Hexahedral FR kernels with a correction function c != 0 of the energy-stable family of
// Vincent, Castonguay & Jameson (2011); the paper (section "FR Algorithm") takes its c = 0,
// DG-equivalent member, which the kernels in fr_kernels.cu serve from constant memory.
//
// Only the 1D correction vectors change with c: hm = g_R'(-x_i), hp = g_R'(x_i) and the
// divergence operator with the own-flux correction folded in, Dt = D - hp (x) lp + hm (x) lm.
// These kernels run the same volume and correction bodies on the mesh's own copy of the tables
// (global memory, read through L1), so the c = 0 kernels keep their constant-memory tables
// untouched.  Interpolation and interface kernels do not depend on c and are shared.
#include "fr_bodies.cuh"

namespace frx {

template <int N, typename T>
__global__ void __launch_bounds__(volume_threads<N>(), volume_min_blocks<N>())
    k_volume_vc(const T *__restrict__ Q, const T *__restrict__ metrics, const int32_t *__restrict__ ef,
                const T *__restrict__ Qtr, const T *__restrict__ liftfac, T *__restrict__ Gtr, T *__restrict__ Rpart,
                DevPhys dph, const double *__restrict__ hel, float *__restrict__ nu_out,
                const int8_t *__restrict__ if_up, int64_t n_interior) {
  extern __shared__ double sm_raw[];
  volume_body<N, T, true>(blockIdx.x, threadIdx.x, blockDim.x, true, sm_raw, Q, metrics, ef, Qtr, liftfac, Gtr,
                          Rpart, dph, hel, nu_out, if_up, n_interior);
}

template <int N, typename T>
__global__ void k_correct_vc(const T *__restrict__ Rpart, const T *__restrict__ FI, const int32_t *__restrict__ ef,
                             const T *__restrict__ metrics, int64_t E, int mode, int stage, double dt,
                             double *__restrict__ Rout, double *__restrict__ Q, T *__restrict__ Qc,
                             double *__restrict__ Un, T *__restrict__ Unc, double *__restrict__ acc,
                             int *__restrict__ flag, DevPhys dph) {
  correct_body<N, T, true>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, Rpart, FI, ef, metrics, E, mode, stage,
                           dt, Rout, Q, Qc, Un, Unc, acc, flag, dph);
}

template <int N, typename T>
static cudaError_t vcjh_phase_impl(const DevMesh &m, const DevPhys &ph, int phase, int mode, int stage, double dt,
                                   double *Rout, cudaStream_t st) {
  constexpr int Np = N * N * N, Nf = N * N;
  const int64_t E = m.E;
  if (E == 0) return cudaSuccess;
  if (!ph.vc_basis || m.Ep != 0) return cudaErrorInvalidValue;
  const T *Qin = reinterpret_cast<const T *>(m.mixed ? m.Qc : m.Q);
  T *Gtr = reinterpret_cast<T *>(m.Gtr), *FI = reinterpret_cast<T *>(m.FI);
  T *Rpart = reinterpret_cast<T *>(m.Rpart);
  const T *met = reinterpret_cast<const T *>(m.metrics);
  if (phase == 1) {
    const size_t smem = sizeof(T) * (35 * Np + 30 * Nf) + (ph.closure ? sizeof(float) * (10 * Np + 1 + 128) : 0);
    cudaError_t err = cudaFuncSetAttribute(k_volume_vc<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_volume_vc<N, T><<<(unsigned)E, volume_threads<N>(), smem, st>>>(
        Qin, met, m.ef, reinterpret_cast<const T *>(m.Qtr), reinterpret_cast<const T *>(m.liftfac), Gtr, Rpart, ph,
        m.h, m.nu, m.if_up, m.n_interior);
  } else if (phase == 3) {
    const int64_t n = E * Np;
    k_correct_vc<N, T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        Rpart, FI, m.ef, met, E, mode, stage, dt, Rout, m.Q, m.mixed ? reinterpret_cast<T *>(m.Qc) : nullptr, m.Un,
        reinterpret_cast<T *>(m.Unc), m.acc, m.flag, ph);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t vcjh_dispatch(const DevMesh &m, const DevPhys &ph, int phase, int mode, int stage, double dt,
                                 double *Rout, cudaStream_t st) {
  switch (m.N) {
    case 2: return vcjh_phase_impl<2, T>(m, ph, phase, mode, stage, dt, Rout, st);
    case 3: return vcjh_phase_impl<3, T>(m, ph, phase, mode, stage, dt, Rout, st);
    case 4: return vcjh_phase_impl<4, T>(m, ph, phase, mode, stage, dt, Rout, st);
    case 5: return vcjh_phase_impl<5, T>(m, ph, phase, mode, stage, dt, Rout, st);
    case 6: return vcjh_phase_impl<6, T>(m, ph, phase, mode, stage, dt, Rout, st);
    case 7: return vcjh_phase_impl<7, T>(m, ph, phase, mode, stage, dt, Rout, st);
    case 8: return vcjh_phase_impl<8, T>(m, ph, phase, mode, stage, dt, Rout, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_vcjh_phase(const DevMesh &m, const DevPhys &ph, int phase, int mode, int stage, double dt,
                              double *Rout, cudaStream_t st) {
  if (m.mixed) return vcjh_dispatch<df32>(m, ph, phase, mode, stage, dt, Rout, st);
  return vcjh_dispatch<double>(m, ph, phase, mode, stage, dt, Rout, st);
}

cudaError_t vcjh_basis_create(int p, double c, int mixed, void **out) {
  *out = nullptr;
  BasisT<double> d;
  BasisT<df32> f;
  fill_basis(make_basis(p, c), d, f);
  const size_t bytes = mixed ? sizeof(f) : sizeof(d);
  cudaError_t e = cudaMalloc(out, bytes);
  if (e != cudaSuccess) {
    *out = nullptr;
    return e;
  }
  e = cudaMemcpy(*out, mixed ? static_cast<const void *>(&f) : static_cast<const void *>(&d), bytes,
                 cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(*out);
    *out = nullptr;
  }
  return e;
}

}  // namespace frx
