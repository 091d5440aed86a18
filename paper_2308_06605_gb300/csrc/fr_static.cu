// Residual evaluation with library-owned static scratch: the entry point fr_residual_static
// allocates nothing.  Its intermediate arrays (solution traces, gradient traces, common fluxes
// and the partial residual) live in one file-scope device array of fixed size instead of the
// buffers fr_mesh_create allocated; the caller supplies the state and the output.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "fr_device.hpp"

using namespace frx;

namespace {

// 32 MiB of doubles, resident on every device that loads this library until the process exits.
constexpr size_t kStaticScratchDoubles = (size_t(32) << 20) / sizeof(double);
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the static array on the current device, looked up once per device.
cudaError_t scratch_address(int device, double **out) {
  std::lock_guard<std::mutex> lk(g_setup_mutex);
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_scratch_addr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" fr_status fr_residual_static(fr_mesh *mesh, const double *Q_device, double *R_device) {
  DevMesh dev;
  DevPhys phys;
  cudaStream_t stream;
  int device = 0;
  fr_status st = frx_mesh_view(mesh, &dev, &phys, &stream, &device);
  if (st != FR_OK) return st;
  if (!Q_device || !R_device) return frx_mesh_fail(mesh, FR_EINVAL, "fr_residual_static: NULL state or residual");
  if (dev.mixed) return frx_mesh_fail(mesh, FR_EUNSUPPORTED, "fr_residual_static: FP64 meshes only");
  if (dev.Ep > 0) return frx_mesh_fail(mesh, FR_EUNSUPPORTED, "fr_residual_static: hexahedral meshes only");
  if (frx_mesh_has_halo(mesh))
    return frx_mesh_fail(mesh, FR_EUNSUPPORTED, "fr_residual_static: parts that share interfaces with other parts");
  if (phys.vc_basis)
    return frx_mesh_fail(mesh, FR_EUNSUPPORTED, "fr_residual_static: DG-equivalent correction (c = 0) only");
  // The closure writes each element's eddy viscosity into a mesh-owned array, which would make
  // this call change the mesh; it is refused instead.
  if (phys.closure)
    return frx_mesh_fail(mesh, FR_EUNSUPPORTED, "fr_residual_static: meshes without the eddy-viscosity closure only");
  const size_t Nf = (size_t)dev.Nf;
  const size_t n_qtr = (size_t)dev.n_if * 2 * 5 * Nf;
  const size_t n_gtr = (size_t)dev.n_if * 2 * 15 * Nf;
  const size_t n_fi = (size_t)dev.n_if * 5 * Nf;
  const size_t n_rp = (size_t)dev.E * dev.Np * 5;
  const size_t need = n_qtr + n_gtr + n_fi + n_rp;
  if (need > kStaticScratchDoubles) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "fr_residual_static: mesh needs %zu bytes of scratch, the static array holds %zu bytes",
             need * sizeof(double), kStaticScratchDoubles * sizeof(double));
    return frx_mesh_fail(mesh, FR_EINVAL, buf);
  }
  int current = -1;
  cudaError_t e = cudaGetDevice(&current);
  if (e == cudaSuccess && current != device) {
    // A caller error, not a failed CUDA call: nothing ran, so the mesh stays usable.
    char buf[160];
    snprintf(buf, sizeof buf, "fr_residual_static: current device %d differs from the mesh's device %d", current,
             device);
    return frx_mesh_fail(mesh, FR_EINVAL, buf);
  }
  double *base = nullptr;
  if (e == cudaSuccess) e = scratch_address(device, &base);
  if (e != cudaSuccess)
    return frx_mesh_fail(mesh, FR_ECUDA, std::string("fr_residual_static: ") + cudaGetErrorString(e));
  // Every array below is fully written by the kernel that produces it before it is read, so
  // nothing left by an earlier call needs clearing.
  dev.Q = const_cast<double *>(Q_device);   // read only in residual mode
  dev.Qtr = base;
  dev.Gtr = dev.Qtr + n_qtr;
  dev.FI = dev.Gtr + n_gtr;
  dev.Rpart = dev.FI + n_fi;
  e = launch_residual(dev, phys, MODE_RESIDUAL, 0, 0.0, R_device, stream, nullptr);
  if (e != cudaSuccess)
    return frx_mesh_fail(mesh, FR_ECUDA, std::string("fr_residual_static: ") + cudaGetErrorString(e));
  return FR_OK;
}
