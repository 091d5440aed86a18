// Internal declarations shared by the host builder, the kernels and the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "fr.h"

namespace frx {

constexpr int kMaxN = 8;      // p <= 7
constexpr int kMaxBC = 32;    // distinct boundary conditions per mesh

// 1D arrays of the order-p Gauss-Legendre element, computed in long double.
struct Basis1D {
  int p = 0, N = 0;
  double x[kMaxN], w[kMaxN];
  double D[kMaxN * kMaxN];       // D[i*N + a] = l_a'(x_i)
  double lm[kMaxN], lp[kMaxN];   // l_a(-1), l_a(+1)
  double hm[kMaxN], hp[kMaxN];   // correction divergence on the normal line of the -/+ face
};
Basis1D make_basis(int p);

// Connectivity + geometry, host side, before upload.
struct HostMesh {
  int p = 0, N = 0, Np = 0, Nf = 0;
  int64_t E = 0;
  int64_t n_if = 0;               // interfaces (interior + periodic) followed by boundary faces
  int64_t n_interior = 0;         // first n_interior entries are two-sided
  std::vector<int32_t> ef;        // [E][6] packed: (iface << 4) | (side << 3) | orient
  std::vector<int32_t> if_bc;     // [n_if] -1 two-sided, else index into bcs
  std::vector<int32_t> if_elem;   // [n_if][2] element of side 0 and side 1 (-1 for a boundary)
  std::vector<double> metrics;    // [E][10][Np]: S (row-major d, j) then 1/|J|
  std::vector<double> liftfac;    // [E][6][3][Nf]
  std::vector<double> normals;    // [n_if][4][Nf] outward area-scaled normal of side 0, then |n|
  std::vector<double> xsol;       // [E][Np][3]
  std::vector<double> h;          // [E] volume^(1/3)
  std::vector<fr_bc> bcs;
};

fr_status build_host_mesh(const fr_mesh_desc *d, HostMesh &m, std::string &err);

// Slot (side-0 ordering) of the local face point (a, b) for an orientation code.
inline int orient_slot(int code, int a, int b, int N) {
  if (code & 4) { int t = a; a = b; b = t; }
  if (code & 1) a = N - 1 - a;
  if (code & 2) b = N - 1 - b;
  return a + N * b;
}

}  // namespace frx
