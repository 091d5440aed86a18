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
  T gamma, gm1, cT, mu, m2mu3, kappa, eta;   // cT = (gamma-1)/R, m2mu3 = -2 mu / 3; eta = 0 for LDG
  T zero, half, one;
  T tau;                                     // LDG penalty
};

struct DevPhys {
  double gamma, R, mu, kappa, eta;
  int viscous;
  int ldg;                 // viscous scheme: 0 BR2, 1 LDG
  double ldg_tau;
  int inviscid;
  int closure;             // eddy-viscosity network on (weights below)
  double cp_prt;           // cp / Pr_t
  const void *cw;          // [9153] bf16 network parameters (device)
  const float *cscale;     // [23] input mean (11), input std (11), output scale (device)
  PhysT<double> d;
  PhysT<df32> f;
  PhysT<float> s;          // the viscous branch of the double-float path
  // Source term S of Eq. 3 (fr_set_source): body acceleration and sponge, FP64.
  int src_body, src_sponge;
  double accel[3];
  const double *sigma;     // [n_points] device
  const double *Q_ref;     // [n_points][5] device
  // Correction function c != 0 of the energy-stable family: the mesh's 1D tables (a BasisT of
  // the element arithmetic, device); null for the DG-equivalent tables in constant memory.
  const void *vc_basis;
};

// Device buffers of one mesh (all owned by the mesh).
struct DevMesh {
  int p, N, Np, Nf;
  int64_t E, n_if, n_interior;
  int mixed;        // 1: element arrays hold df32 pairs (same 8-byte slots), Qc holds the state as df32
  int tc;           // 1 (mixed only): face interpolation on the tensor cores (FR_PREC_MIXED_TC)
  int vf32;         // 1 (mixed only): viscous branch of the volume kernel in FP32 (FR_PREC_MIXED_VF32)
  double *Q, *Un, *acc, *Rpart, *metrics, *liftfac, *normals, *Qtr, *Gtr, *FI, *h, *dtbuf, *Qc, *Unc;
  int32_t *ef, *if_bc;
  int32_t *if_elem;        // [n_if][2] element of each side (-1: boundary), closure only
  float *nu;               // [E] eddy viscosity of each element, closure only
  fr_bc *bcs;
  int *flag;
  // Prisms (after the E hexahedra in Q, Un, acc, Rpart, Qc, Unc, h); zero / null on hexahedral meshes.
  int64_t Ep;
  int Nt, Npp;             // triangle nodes, points per prism
  int32_t *ef_p;           // [Ep][5] packed like ef (triangular faces: kTriPerm code)
  double *metrics_p;       // [Ep][10][Npp] S then 1/|J|, in the element type
  double *ptab;            // prism operator table (prism_tab layout), in the element type
  int32_t *tri_slot;       // [6][Nt] side-0 slot of a side-1 triangle node per code
  int8_t *if_tri;          // [n_if] 1: triangular interface (only its first Nt slots are used)
  int8_t *if_up;           // [n_if] LDG: 1 if side 0 supplies the common solution, else side 1
};

// What the correction kernels do with the residual: write it, or apply a stage of RK44, of the
// three-stage SSP scheme (Shu-Osher form) or of Ketcheson's ten-stage fourth-order SSP scheme.
enum { MODE_RESIDUAL = 0, MODE_RK = 1, MODE_SSP33 = 2, MODE_SSP104 = 3 };

// Optional per-kernel event pairs (instrumentation); null = off.
struct PhaseEvents {
  cudaEvent_t start[4], stop[4];
};

cudaError_t upload_basis_tables();
// Residual of the current state dev.Q; MODE_RESIDUAL writes R (canonical layout) to Rout,
// MODE_RK applies RK44 stage `stage` with step dt.  `phases` selects the parts that run (bit k:
// 0 face traces and boundary states, 1 volume, 2 interface and boundary fluxes, 3 correction and
// output / stage update), so a domain-decomposed stage can exchange halo traces in between.
cudaError_t launch_residual(const DevMesh &m, const DevPhys &ph, int mode, int stage, double dt,
                            double *Rout, cudaStream_t st, const PhaseEvents *ev = nullptr, int phases = 15);
// ---------------------------------------------------------------- batched persistent stage
// One case of a batch: its device view, physics and precision (all cases share the precision).
struct BatchCase {
  DevMesh m;
  DevPhys ph;
};

// Work item of a phase: case `cs`, kind, and an item range [begin, end) -- flux/solution
// points for the pointwise kinds, elements for the volume kind.
enum { TASK_INTERP = 0, TASK_BC_PREPARE = 1, TASK_VOLUME = 2, TASK_IFACE = 3, TASK_BC_FLUX = 4, TASK_CORRECT = 5,
       TASK_PRISM_INTERP = 6, TASK_PRISM_VOLUME = 7, TASK_PRISM_CORRECT = 8 };
struct BatchTask {
  int32_t cs, kind;
  int64_t begin, end;
};

// Device state of one stage launch: task counters per phase, grid-barrier count/generation,
// error word (1 = a barrier wait gave up), non-finite flag.
struct BatchSync {
  unsigned counters[8];
  unsigned bar_count, bar_gen;
  int err;
  int nonfinite;
};

struct BatchLaunch {
  const BatchCase *cases;
  const BatchTask *tasks;
  int phase_begin[6];    // tasks of phase k are [phase_begin[k], phase_begin[k+1])
  int n_phases;
  int stage;
  const double *dts;     // [n_cases] device
  BatchSync *sync;
  long long spin_limit;  // iterations of a barrier wait before giving up
  int debug_skip_block;  // >= 0: that block leaves before the first barrier (timeout test)
};

// Variants of the batched stage kernel (fr_batch_kernel.cu, compiled once per precision m = 0 FP64,
// 1 double-float and block size b): launch, resident blocks per SM, upload of the unit's basis.
#define FRX_BATCH_VARIANT_DECL(m, b)                                                                    \
  cudaError_t batch_launch_m##m##_b##b(const BatchLaunch &L, int grid, size_t smem, cudaStream_t st); \
  cudaError_t batch_occupancy_m##m##_b##b(size_t smem, int *nb);                                       \
  cudaError_t batch_upload_m##m##_b##b();
FRX_BATCH_VARIANT_DECL(0, 256)
FRX_BATCH_VARIANT_DECL(0, 512)
FRX_BATCH_VARIANT_DECL(1, 256)
FRX_BATCH_VARIANT_DECL(1, 512)
#undef FRX_BATCH_VARIANT_DECL

// Launch one cooperative persistent stage over all cases (block size 256 or 512).
cudaError_t launch_batch_stage(const BatchLaunch &L, int mixed, int block, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_gather_flags(const BatchCase *cases, int n, BatchSync *sy, cudaStream_t st);
// Largest dynamic shared memory one block needs for the given orders (and whether each case has
// prisms) and block size.
size_t batch_smem_bytes(const int *Ns, const int *has_prism, int n, int block, int mixed);
// Resident blocks per SM of the batch kernel for the given configuration.
cudaError_t batch_occupancy(int mixed, int block, size_t smem, int *blocks_per_sm);
// Elements a block of `block` threads processes at once in the volume phase for order N: as many
// sub-blocks of (points rounded up to a warp) threads as fit, capped so that their shared memory
// stays within kBatchSmemBudget bytes.  Host (task lists, shared-memory size) and device (sub-block
// layout) use the same functions.
constexpr int kBatchSmemBudget = 220 * 1024;
FRX_HD inline int batch_fit(int points, int smem_values, int block) {
  const int tpe = ((points + 31) / 32) * 32;
  const int by_threads = tpe >= block ? 1 : block / tpe;
  const int by_smem = kBatchSmemBudget / (smem_values * 8);
  return by_threads < by_smem ? by_threads : (by_smem > 0 ? by_smem : 1);
}
FRX_HD inline int batch_elems_per_block(int N, int block) {
  return batch_fit(N * N * N, 35 * N * N * N + 30 * N * N, block);
}
// The same for prisms (N(N+1)/2 x N points).
FRX_HD inline int batch_prism_elems_per_block(int N, int block) {
  return batch_fit(N * (N + 1) / 2 * N, 65 * (N * (N + 1) / 2 * N) + 25 * N * N, block);
}

// Accessors of the opaque mesh (fr_api.cu): a copy of its device view (fails if poisoned), and
// recording an error on it.
fr_status frx_mesh_view(fr_mesh *m, DevMesh *dev, DevPhys *phys, cudaStream_t *stream, int *device);
fr_status frx_mesh_fail(fr_mesh *m, fr_status st, const std::string &msg);
// True for a part of a domain-decomposed mesh that shares interfaces with other parts.
bool frx_mesh_has_halo(const fr_mesh *m);

// Prism phases of one residual evaluation (fr_prism.cu): 0 face traces, 1 volume, 3 correction
// and output / RK update; a no-op on hexahedral meshes.
cudaError_t launch_prism_phase(const DevMesh &m, const DevPhys &ph, int phase, int mode, int stage, double dt,
                               double *Rout, cudaStream_t st);
// Per-prism time-step bound into m.dtbuf[E + ep] (same formula as the hexahedra).
// Hexahedral volume (phase 1) and correction (phase 3) kernels reading the mesh's own 1D tables
// (correction function c != 0); vcjh_basis_create builds and uploads those tables.
cudaError_t launch_vcjh_phase(const DevMesh &m, const DevPhys &ph, int phase, int mode, int stage, double dt,
                              double *Rout, cudaStream_t st);
cudaError_t vcjh_basis_create(int p, double c, int mixed, void **out);
cudaError_t launch_prism_dt(const DevMesh &m, const DevPhys &ph, double cfl, cudaStream_t st);

// Halo traces of a domain-decomposed mesh (X = Qtr with nv = 5 or Gtr with nv = 15): pack this
// part's slots of the listed interfaces into buf, or unpack buf into the other sides' slots.
cudaError_t launch_halo_copy(double *X, double *buf, const int64_t *code, int64_t n_halo, int nv, int Nf, int unpack,
                             cudaStream_t st);

// Tensor-core face interpolation of the double-float state (fr_tc.cu) and its operator tables.
cudaError_t launch_interp_tc(const DevMesh &m, cudaStream_t st);
cudaError_t upload_tc_tables();

// Mixed path: refresh the df32 copy of the state after it was set from outside.
cudaError_t launch_state_copy(const DevMesh &m, cudaStream_t st);
cudaError_t launch_max_dt(const DevMesh &m, const DevPhys &ph, double cfl, double *d_out, cudaStream_t st);

}  // namespace frx
