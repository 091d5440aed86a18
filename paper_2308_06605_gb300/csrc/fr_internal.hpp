// Internal declarations shared by the host builder, the kernels and the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "fr.h"

#ifdef __CUDACC__
#define FRX_HD __host__ __device__
#else
#define FRX_HD
#endif

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
// Order-p Gauss-Legendre basis; c selects the correction function of the energy-stable family
// (0: DG-equivalent Radau).  The caller checks vcjh_in_family(p, c) first.
Basis1D make_basis(int p, double c = 0.0);
bool vcjh_in_family(int p, double c);

// Nodal triangle basis of order p (prism elements): warp-and-blend nodes, operators from the
// orthonormal Proriol-Koornwinder-Dubiner modes, all computed in long double.
struct TriBasis {
  int p = 0, N = 0, Nt = 0;
  std::vector<double> r, s;        // [Nt] nodes, enumerated n = 0..p (outer), m = 0..p-n (inner)
  std::vector<double> Dr, Ds;      // [Nt][Nt] derivative matrices
  std::vector<double> Minv;        // [Nt][Nt] inverse mass matrix
  std::vector<double> wT;          // [Nt] integral of each nodal function over the triangle
  std::vector<double> E[3];        // [N][Nt] interpolation to the Gauss-Legendre points of edge e
  std::vector<double> LQ[3];       // [Nt][N] DG lifting of edge e: M^-1 E^T diag(w)
  std::vector<int32_t> perm;       // [6][Nt] image node under the vertex permutation kTriPerm[c]
};
extern const int kTriPerm[6][3];
// Point of edge e (0: s = -1, 1: r + s = 0, 2: r = -1) at parameter sigma in [-1, 1].
void tri_edge_point(int edge, double sigma, double &r, double &s);
bool make_tri_basis(int p, TriBasis &T);
// [Nt_q][Nt_p]: the L2 projection from the order-p to the order-q triangle (nodal values in,
// nodal values out; orthonormal modes of total degree <= min(p, q) kept).
bool tri_transfer(int p, int q, std::vector<double> &T);
// p + 1 Gauss-Lobatto-Legendre points (ascending).
void gll_nodes(int p, double *x);

// Quadratic (curved) element geometry (fr_curved.cpp).  1D operators from the p + 1
// Gauss-Lobatto points g to the Gauss-Legendre points x of the line and to its ends.
struct CurvedOps {
  int p = 0, N = 0, Nt = 0;
  double g[kMaxN];
  double V[kMaxN * kMaxN], D[kMaxN * kMaxN];   // [i][a] = l_a(x_i), l_a'(x_i)
  double Ve[2][kMaxN], De[2][kMaxN];           // l_a(-1), l_a'(-1); l_a(+1), l_a'(+1)
  // Quadratic Lagrange functions of the nodes -1, 0, 1 (value, derivative) at the Gauss-Lobatto
  // points [N][3], the Gauss-Legendre points [N][3] and the ends [2][3].
  double Qg[kMaxN * 3], dQg[kMaxN * 3], Qx[kMaxN * 3], dQx[kMaxN * 3], Qe[6], dQe[6];
  // Prisms: the 6 quadratic triangle functions (corners 0 1 2, midpoints 01 12 20) and their r, s
  // derivatives at the triangle nodes [Nt][6] and at the Gauss points of each edge [3][N][6].
  std::vector<double> T, Tr, Ts, TE[3], TEr[3], TEs[3];
};
void curved_ops(int p, const Basis1D &b, const TriBasis *tb, CurvedOps &o);
// Geometry of one quadratic element (node orders as documented in fr.h): position x and |J| at
// the solution points (x_sol [Np][3], det [Np]), the conservative-curl metric terms
// S[(d*3 + j)] = |J| dxi_d/dx_j at the solution points (S_sol [9][Np]), and at the flux points of
// every face the position (x_face [faces][N^2][3]) and the rows of S that make up the face's
// reference normal (S_face [faces][9][N^2]; other rows are left untouched; a triangular face uses
// its first Nt slots).
void hex27_geometry(const CurvedOps &o, const double (*X)[3], double *x_sol, double *det, double *S_sol,
                    double *x_face, double *S_face);
void prism18_geometry(const CurvedOps &o, const TriBasis &tb, const double (*X)[3], double *x_sol, double *det,
                      double *S_sol, double *x_face, double *S_face);

// Offsets (in values) of the per-mesh prism operator table for line order N (Nt = N(N+1)/2):
// Dr, Ds (triangle derivatives), Drt, Dst (with the own-flux correction of the quadrilateral
// faces folded in), E [3][N][Nt], LQ [3][Nt][N], D1, D1t [N][N] (line derivative, plain and with
// the own-flux correction of the triangular faces), then l(-1), l(+1), h-, h+ [N] each.
struct PrismTab {
  int Nt, Dr, Ds, Drt, Dst, E, LQ, D1, D1t, lm, lp, hm, hp, size;
};
FRX_HD constexpr PrismTab prism_tab(int N) {
  const int Nt = N * (N + 1) / 2, T2 = Nt * Nt;
  return PrismTab{Nt,
                  0,
                  T2,
                  2 * T2,
                  3 * T2,
                  4 * T2,
                  4 * T2 + 3 * N * Nt,
                  4 * T2 + 6 * N * Nt,
                  4 * T2 + 6 * N * Nt + N * N,
                  4 * T2 + 6 * N * Nt + 2 * N * N,
                  4 * T2 + 6 * N * Nt + 2 * N * N + N,
                  4 * T2 + 6 * N * Nt + 2 * N * N + 2 * N,
                  4 * T2 + 6 * N * Nt + 2 * N * N + 3 * N,
                  4 * T2 + 6 * N * Nt + 2 * N * N + 4 * N};
}

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
  std::vector<double> xsol;       // [E][Np][3] then [Ep][Npp][3]
  std::vector<double> h;          // [E + Ep] volume^(1/3)
  std::vector<fr_bc> bcs;
  // Prisms (after the hexahedra in every per-point array).
  int64_t Ep = 0;
  int Nt = 0, Npp = 0;            // triangle nodes, points per prism (Nt * N)
  std::vector<int32_t> ef_p;      // [Ep][5] packed like ef; triangular faces carry a kTriPerm code
  std::vector<double> metrics_p;  // [Ep][10][Npp]
  std::vector<int8_t> if_tri;     // [n_if] 1: triangular interface (meshes with prisms only)
  std::vector<int8_t> if_up;      // [n_if] LDG switch: 1 if side 0 supplies the common solution
  std::vector<double> ptab;       // prism operator table (prism_tab layout)
  std::vector<int32_t> tri_slot;  // [6][Nt] side-0 slot of a side-1 node for each code
};

fr_status build_host_mesh(const fr_mesh_desc *d, HostMesh &m, std::string &err, double vcjh_c = 0.0);

// Slot (side-0 ordering) of the local face point (a, b) for an orientation code.
FRX_HD inline int orient_slot(int code, int a, int b, int N) {
  if (code & 4) { int t = a; a = b; b = t; }
  if (code & 1) a = N - 1 - a;
  if (code & 2) b = N - 1 - b;
  return a + N * b;
}

}  // namespace frx
