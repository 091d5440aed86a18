// Projection of a solution between orders (include/fr.h, fr_project_state).  The paper starts its
// runs at low order and switches to a higher one; the state is carried over by the L2 projection
// onto the target space in reference coordinates: Legendre modal coefficients on each hexahedron
// axis (truncated or zero-padded), the orthonormal triangle modes times Legendre on the prism.
// A one-off operation: one thread per target point, FP64, 1D operators from the host.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "fr_device.hpp"

namespace frx {
namespace {

// [q+1][p+1]: the line transfer through the Gauss points, with the exact discrete orthogonality
// of the Legendre polynomials on the order-p Gauss rule (c_k = (2k+1)/2 sum_j w_j P_k(x_j) f_j).
void line_transfer(int p, int q, std::vector<double> &T) {
  const Basis1D bp = make_basis(p), bq = make_basis(q);
  const int m = (p < q ? p : q) + 1;
  auto legendre = [](long double x, int n, long double *P) {
    P[0] = 1.0L;
    if (n > 0) P[1] = x;
    for (int k = 1; k < n; ++k) P[k + 1] = ((2 * k + 1) * x * P[k] - k * P[k - 1]) / (k + 1);
  };
  T.assign((size_t)(q + 1) * (p + 1), 0.0);
  long double Pp[kMaxN + 1], Pq[kMaxN + 1];
  for (int i = 0; i <= q; ++i) {
    legendre((long double)bq.x[i], kMaxN, Pq);
    for (int j = 0; j <= p; ++j) {
      legendre((long double)bp.x[j], kMaxN, Pp);
      long double acc = 0.0L;
      for (int k = 0; k < m; ++k) acc += Pq[k] * (2 * k + 1) / 2.0L * (long double)bp.w[j] * Pp[k];
      T[(size_t)i * (p + 1) + j] = (double)acc;
    }
  }
}

// Hexahedra: out(i, j, k) = sum L[i][a] L[j][b] L[k][c] in(a, b, c); prisms:
// out(t, k) = sum L[k][c] Tt[t][s] in(s, c).  Np/Nq: points per element of source / target.
__global__ void k_project(const double *__restrict__ src, double *__restrict__ dst, const double *__restrict__ L,
                          const double *__restrict__ Tt, int64_t n_elem, int Ns, int Nd, int Nts, int Ntd, int prism) {
  const int Nq = prism ? Ntd * Nd : Nd * Nd * Nd, Np = prism ? Nts * Ns : Ns * Ns * Ns;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_elem * Nq) return;
  const int64_t e = t / Nq;
  const int m = (int)(t % Nq);
  const double *in = src + e * Np * 5;
  double acc[5] = {0, 0, 0, 0, 0};
  if (!prism) {
    const int i = m % Nd, j = (m / Nd) % Nd, k = m / (Nd * Nd);
    for (int c = 0; c < Ns; ++c)
      for (int b = 0; b < Ns; ++b) {
        const double wbc = L[k * Ns + c] * L[j * Ns + b];
        for (int a = 0; a < Ns; ++a) {
          const double w = wbc * L[i * Ns + a];
          const double *q = in + (a + Ns * (b + Ns * c)) * 5;
          for (int v = 0; v < 5; ++v) acc[v] += w * q[v];
        }
      }
  } else {
    const int tt = m % Ntd, k = m / Ntd;
    for (int c = 0; c < Ns; ++c)
      for (int s = 0; s < Nts; ++s) {
        const double w = L[k * Ns + c] * Tt[tt * Nts + s];
        const double *q = in + (s + Nts * c) * 5;
        for (int v = 0; v < 5; ++v) acc[v] += w * q[v];
      }
  }
  for (int v = 0; v < 5; ++v) dst[(e * Nq + m) * 5 + v] = acc[v];
}

}  // namespace
}  // namespace frx

using namespace frx;

extern "C" fr_status fr_transfer_matrix(int32_t kind, int32_t p, int32_t q, double *T) {
  if (!T || p < 1 || p > 7 || q < 1 || q > 7 || (kind != 0 && kind != 1)) return FR_EINVAL;
  std::vector<double> M;
  if (kind == 0)
    line_transfer(p, q, M);
  else if (!tri_transfer(p, q, M))
    return FR_EINVAL;
  for (size_t i = 0; i < M.size(); ++i) T[i] = M[i];
  return FR_OK;
}

extern "C" fr_status fr_project_state(fr_mesh *src, fr_mesh *dst) {
  DevMesh a, b;
  DevPhys pa, pb;
  cudaStream_t sa, sb;
  int da = 0, db = 0;
  fr_status st = frx_mesh_view(src, &a, &pa, &sa, &da);
  if (st != FR_OK) return st;
  st = frx_mesh_view(dst, &b, &pb, &sb, &db);
  if (st != FR_OK) return st;
  if (da != db) return frx_mesh_fail(dst, FR_EINVAL, "fr_project_state: meshes on different devices");
  if (a.E != b.E || a.Ep != b.Ep)
    return frx_mesh_fail(dst, FR_EINVAL, "fr_project_state: the meshes must have the same elements");
  std::vector<double> L, Tt;
  line_transfer(a.p, b.p, L);
  if (a.Ep > 0 && !tri_transfer(a.p, b.p, Tt))
    return frx_mesh_fail(dst, FR_EMESH, "fr_project_state: triangle transfer failed");
  double *dL = nullptr, *dT = nullptr;
  cudaError_t e = cudaMalloc((void **)&dL, L.size() * sizeof(double));
  if (e == cudaSuccess && !Tt.empty()) e = cudaMalloc((void **)&dT, Tt.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamSynchronize(sa);   // the source state is complete
  if (e == cudaSuccess) e = cudaMemcpyAsync(dL, L.data(), L.size() * sizeof(double), cudaMemcpyHostToDevice, sb);
  if (e == cudaSuccess && dT) e = cudaMemcpyAsync(dT, Tt.data(), Tt.size() * sizeof(double), cudaMemcpyHostToDevice, sb);
  if (e == cudaSuccess && a.E > 0) {
    const int64_t n = b.E * b.Np;
    k_project<<<(unsigned)((n + 255) / 256), 256, 0, sb>>>(a.Q, b.Q, dL, nullptr, a.E, a.N, b.N, 0, 0, 0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && a.Ep > 0) {
    const int64_t n = b.Ep * b.Npp;
    k_project<<<(unsigned)((n + 255) / 256), 256, 0, sb>>>(a.Q + a.E * a.Np * 5, b.Q + b.E * b.Np * 5, dL, dT, a.Ep,
                                                           a.N, b.N, a.Nt, b.Nt, 1);
    e = cudaGetLastError();
  }
  // The projected state starts a new step, as after fr_set_state.
  const size_t bytes = ((size_t)b.E * b.Np + (size_t)b.Ep * b.Npp) * 5 * sizeof(double);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b.Un, b.Q, bytes, cudaMemcpyDeviceToDevice, sb);
  if (e == cudaSuccess) e = launch_state_copy(b, sb);
  if (e == cudaSuccess) e = cudaStreamSynchronize(sb);
  if (dL) cudaFree(dL);
  if (dT) cudaFree(dT);
  if (e != cudaSuccess) return frx_mesh_fail(dst, FR_ECUDA, std::string("fr_project_state: ") + cudaGetErrorString(e));
  return FR_OK;
}
