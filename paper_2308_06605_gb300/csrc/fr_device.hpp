// Device-side declarations: basis tables in constant memory and kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "df32.cuh"
#include "fr_internal.hpp"

namespace frx {

// Physical constants in the element arithmetic's scalar type (double or df32).
template <typename T>
struct PhysT {
  T gamma, gm1, cT, mu, m2mu3, kappa, eta;   // cT = (gamma-1)/R, m2mu3 = -2 mu / 3
  T zero, half, one;
};

struct DevPhys {
  double gamma, R, mu, kappa, eta;
  int viscous;
  int inviscid;
  PhysT<double> d;
  PhysT<df32> f;
};

// Device buffers of one mesh (all owned by the mesh).
struct DevMesh {
  int p, N, Np, Nf;
  int64_t E, n_if, n_interior;
  int mixed;        // 1: element arrays hold df32 pairs (same 8-byte slots), Qc holds the state as df32
  double *Q, *Un, *acc, *Rpart, *metrics, *liftfac, *normals, *Qtr, *Gtr, *FI, *h, *dtbuf, *Qc, *Unc;
  int32_t *ef, *if_bc;
  fr_bc *bcs;
  int *flag;
};

enum { MODE_RESIDUAL = 0, MODE_RK = 1 };

// Optional per-kernel event pairs (instrumentation); null = off.
struct PhaseEvents {
  cudaEvent_t start[4], stop[4];
};

cudaError_t upload_basis_tables();
// Residual of the current state dev.Q; MODE_RESIDUAL writes R (canonical layout) to Rout,
// MODE_RK applies RK44 stage `stage` with step dt.
cudaError_t launch_residual(const DevMesh &m, const DevPhys &ph, int mode, int stage, double dt,
                            double *Rout, cudaStream_t st, const PhaseEvents *ev = nullptr);
// Accessors of the opaque mesh (fr_api.cu): a copy of its device view (fails if poisoned), and
// recording an error on it.
fr_status frx_mesh_view(fr_mesh *m, DevMesh *dev, DevPhys *phys, cudaStream_t *stream, int *device);
fr_status frx_mesh_fail(fr_mesh *m, fr_status st, const std::string &msg);

// Mixed path: refresh the df32 copy of the state after it was set from outside.
cudaError_t launch_state_copy(const DevMesh &m, cudaStream_t st);
cudaError_t launch_max_dt(const DevMesh &m, const DevPhys &ph, double cfl, double *d_out, cudaStream_t st);

}  // namespace frx
