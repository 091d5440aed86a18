// Quadratic (curved) element geometry: element maps and conservative-curl metric terms.
//
// The FR metric terms (section "FR Algorithm", Eq. 1: S = |J| J^-1) of a curved element are taken
// from the conservative curl form of Kopriva (2006): with (n, m, l) cyclic,
//     S[i][n] = -( curl_xi  I(X_l grad_xi X_m) )_i ,
// where I is the degree-p interpolant on a node set that contains the element's faces -- the
// Gauss-Lobatto points on each hexahedron axis, the triangle's warp-and-blend nodes times
// Gauss-Lobatto points in zeta on the prism.  S is then a polynomial of degree p, evaluated
// exactly at the solution points and at the flux points: the discrete metric identities hold and
// a face's normal depends only on the face's own geometry, so both sides of an interface agree and
// uniform flow stays uniform to rounding.  For p >= 2 the interpolant reproduces grad X_m (degree
// <= 2), so measuring X_l from the element's corner centroid leaves S unchanged; it is done to keep
// coordinates small against the element.  Derivatives of the interpolant at the targets are
// applied one axis at a time (1D Lagrange matrices from the Gauss-Lobatto points; the triangle's
// nodal derivative and edge-interpolation matrices).
#include <cmath>
#include <vector>

#include "fr_internal.hpp"

namespace frx {

using ld = long double;

namespace {

// Reference coordinates of the quadratic elements' nodes (node orders as documented in fr.h).
const int kHex27[27][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1}, {-1, -1, 1}, {1, -1, 1}, {1, 1, 1},
                           {-1, 1, 1},   {0, -1, -1}, {1, 0, -1}, {0, 1, -1},  {-1, 0, -1}, {0, -1, 1}, {1, 0, 1},
                           {0, 1, 1},    {-1, 0, 1},  {-1, -1, 0}, {1, -1, 0}, {1, 1, 0},   {-1, 1, 0}, {-1, 0, 0},
                           {1, 0, 0},    {0, -1, 0},  {0, 1, 0},  {0, 0, -1},  {0, 0, 1},   {0, 0, 0}};
// Prism: (triangle node code, zeta level); triangle codes 0..2 corners, 3..5 midpoints of 01 12 20.
const int kPrism18[18][2] = {{0, -1}, {1, -1}, {2, -1}, {0, 1}, {1, 1}, {2, 1}, {3, -1}, {4, -1}, {5, -1},
                             {3, 1},  {4, 1},  {5, 1},  {0, 0}, {1, 0}, {2, 0}, {3, 0},  {4, 0},  {5, 0}};

inline void quad1d(double t, int c, double &L, double &dL) {
  if (c < 0) { L = 0.5 * t * (t - 1.0); dL = t - 0.5; }
  else if (c > 0) { L = 0.5 * t * (t + 1.0); dL = t + 0.5; }
  else { L = 1.0 - t * t; dL = -2.0 * t; }
}

// Lagrange polynomial a of the nodes g (n of them) and its derivative at x (product formulas).
void lagrange(const double *g, int n, int a, ld x, ld &L, ld &dL) {
  L = 1.0L;
  dL = 0.0L;
  for (int b = 0; b < n; ++b)
    if (b != a) L *= (x - (ld)g[b]) / ((ld)g[a] - (ld)g[b]);
  for (int c = 0; c < n; ++c) {
    if (c == a) continue;
    ld t = 1.0L / ((ld)g[a] - (ld)g[c]);
    for (int b = 0; b < n; ++b)
      if (b != a && b != c) t *= (x - (ld)g[b]) / ((ld)g[a] - (ld)g[b]);
    dL += t;
  }
}

// out[i0 + M0 i1 + M0 M1 i2] = sum A0[i0][a] A1[i1][b] A2[i2][c] f[a + N b + N^2 c].
void apply3(const double *f, int N, const double *A0, int M0, const double *A1, int M1, const double *A2, int M2,
            double *out) {
  std::vector<double> t1((size_t)M0 * N * N), t2((size_t)M0 * M1 * N);
  for (int c = 0; c < N; ++c)
    for (int b = 0; b < N; ++b)
      for (int i = 0; i < M0; ++i) {
        double s = 0.0;
        for (int a = 0; a < N; ++a) s += A0[i * N + a] * f[a + N * b + N * N * c];
        t1[i + (size_t)M0 * (b + (size_t)N * c)] = s;
      }
  for (int c = 0; c < N; ++c)
    for (int j = 0; j < M1; ++j)
      for (int i = 0; i < M0; ++i) {
        double s = 0.0;
        for (int b = 0; b < N; ++b) s += A1[j * N + b] * t1[i + (size_t)M0 * (b + (size_t)N * c)];
        t2[i + (size_t)M0 * (j + (size_t)M1 * c)] = s;
      }
  for (int k = 0; k < M2; ++k)
    for (int j = 0; j < M1; ++j)
      for (int i = 0; i < M0; ++i) {
        double s = 0.0;
        for (int c = 0; c < N; ++c) s += A2[k * N + c] * t2[i + (size_t)M0 * (j + (size_t)M1 * c)];
        out[i + (size_t)M0 * (j + (size_t)M1 * k)] = s;
      }
}

// out[t + T z] = sum_q sum_k A[t][q] Z[z][k] f[q + Nt k]  (triangle part, then zeta part).
void apply_tz(const double *f, int Nt, int N, const double *A, int T, const double *Z, int M, double *out) {
  std::vector<double> t1((size_t)T * N);
  for (int k = 0; k < N; ++k)
    for (int t = 0; t < T; ++t) {
      double s = 0.0;
      for (int q = 0; q < Nt; ++q) s += A[(size_t)t * Nt + q] * f[q + (size_t)Nt * k];
      t1[t + (size_t)T * k] = s;
    }
  for (int z = 0; z < M; ++z)
    for (int t = 0; t < T; ++t) {
      double s = 0.0;
      for (int k = 0; k < N; ++k) s += Z[z * N + k] * t1[t + (size_t)T * k];
      out[t + (size_t)T * z] = s;
    }
}

// v[(n*3 + k)*nn + node] = (X_l - c_l) dX_m/dxi_k at the interpolation nodes, (n, m, l) cyclic.
template <typename PointFn>
void curl_fields(int p, int nn, int n_corner, const double (*X)[3], PointFn at_node, std::vector<double> &v) {
  double c[3] = {0.0, 0.0, 0.0};
  if (p >= 2)
    for (int a = 0; a < n_corner; ++a)
      for (int i = 0; i < 3; ++i) c[i] += X[a][i] / n_corner;
  v.assign((size_t)9 * nn, 0.0);
  for (int node = 0; node < nn; ++node) {
    double x[3], J[3][3];
    at_node(node, x, J);
    for (int n = 0; n < 3; ++n) {
      const int m = (n + 1) % 3, l = (n + 2) % 3;
      for (int k = 0; k < 3; ++k) v[(size_t)(n * 3 + k) * nn + node] = (x[l] - c[l]) * J[m][k];
    }
  }
}

}  // namespace

void curved_ops(int p, const Basis1D &b, CurvedOps &o) {
  const int N = p + 1;
  o.p = p;
  o.N = N;
  gll_nodes(p, o.g);
  for (int i = 0; i < N; ++i)
    for (int a = 0; a < N; ++a) {
      ld L, dL;
      lagrange(o.g, N, a, (ld)b.x[i], L, dL);
      o.V[i * N + a] = (double)L;
      o.D[i * N + a] = (double)dL;
    }
  for (int e = 0; e < 2; ++e)
    for (int a = 0; a < N; ++a) {
      ld L, dL;
      lagrange(o.g, N, a, e ? 1.0L : -1.0L, L, dL);
      o.Ve[e][a] = (double)L;
      o.De[e][a] = (double)dL;
    }
}

void hex27_point(const double (*X)[3], const double xi[3], double x[3], double J[3][3]) {
  for (int i = 0; i < 3; ++i) {
    x[i] = 0.0;
    for (int b = 0; b < 3; ++b) J[i][b] = 0.0;
  }
  for (int a = 0; a < 27; ++a) {
    double L[3], dL[3];
    for (int d = 0; d < 3; ++d) quad1d(xi[d], kHex27[a][d], L[d], dL[d]);
    const double Nv = L[0] * L[1] * L[2];
    const double dN[3] = {dL[0] * L[1] * L[2], L[0] * dL[1] * L[2], L[0] * L[1] * dL[2]};
    for (int i = 0; i < 3; ++i) {
      x[i] += Nv * X[a][i];
      for (int b = 0; b < 3; ++b) J[i][b] += dN[b] * X[a][i];
    }
  }
}

void prism18_point(const double (*X)[3], const double xi[3], double x[3], double J[3][3]) {
  const double r = xi[0], s = xi[1];
  const double lam[3] = {-(r + s) / 2, (1 + r) / 2, (1 + s) / 2};
  const double dlr[3] = {-0.5, 0.5, 0.0}, dls[3] = {-0.5, 0.0, 0.5};
  const int mid[3][2] = {{0, 1}, {1, 2}, {2, 0}};
  for (int i = 0; i < 3; ++i) {
    x[i] = 0.0;
    for (int b = 0; b < 3; ++b) J[i][b] = 0.0;
  }
  for (int a = 0; a < 18; ++a) {
    const int t = kPrism18[a][0];
    double T, Tr, Ts;
    if (t < 3) {             // corner: lambda (2 lambda - 1)
      T = lam[t] * (2 * lam[t] - 1);
      Tr = (4 * lam[t] - 1) * dlr[t];
      Ts = (4 * lam[t] - 1) * dls[t];
    } else {                 // edge midpoint: 4 lambda_i lambda_j
      const int i = mid[t - 3][0], j = mid[t - 3][1];
      T = 4 * lam[i] * lam[j];
      Tr = 4 * (dlr[i] * lam[j] + lam[i] * dlr[j]);
      Ts = 4 * (dls[i] * lam[j] + lam[i] * dls[j]);
    }
    double Z, dZ;
    quad1d(xi[2], kPrism18[a][1], Z, dZ);
    const double Nv = T * Z, dN[3] = {Tr * Z, Ts * Z, T * dZ};
    for (int i = 0; i < 3; ++i) {
      x[i] += Nv * X[a][i];
      for (int b = 0; b < 3; ++b) J[i][b] += dN[b] * X[a][i];
    }
  }
}

void hex27_curl(const CurvedOps &o, const double (*X)[3], double *S_sol, double *S_face) {
  const int N = o.N, N3 = N * N * N, Nf = N * N;
  std::vector<double> v;
  curl_fields(o.p, N3, 8, X, [&](int node, double x[3], double J[3][3]) {
    const double xi[3] = {o.g[node % N], o.g[(node / N) % N], o.g[node / Nf]};
    hex27_point(X, xi, x, J);
  }, v);
  std::vector<double> A(N3), B(N3);
  // Solution points: the Gauss-Legendre tensor grid.
  for (int n = 0; n < 3; ++n)
    for (int i = 0; i < 3; ++i) {
      const int j = (i + 1) % 3, k = (i + 2) % 3;
      const double *M[3];
      for (int d = 0; d < 3; ++d) M[d] = d == j ? o.D : o.V;
      apply3(&v[(size_t)(n * 3 + k) * N3], N, M[0], N, M[1], N, M[2], N, A.data());
      for (int d = 0; d < 3; ++d) M[d] = d == k ? o.D : o.V;
      apply3(&v[(size_t)(n * 3 + j) * N3], N, M[0], N, M[1], N, M[2], N, B.data());
      for (int m = 0; m < N3; ++m) S_sol[(size_t)(i * 3 + n) * N3 + m] = -(A[m] - B[m]);
    }
  // Faces: axis d at its end s, the tangential axes on the Gauss-Legendre points.
  for (int f = 0; f < 6; ++f) {
    const int d = f / 2, e = f % 2;
    for (int n = 0; n < 3; ++n)
      for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3, k = (i + 2) % 3;
        const double *M[3];
        int Ms[3];
        for (int q = 0; q < 3; ++q) {
          Ms[q] = q == d ? 1 : N;
          M[q] = q == d ? (q == j ? o.De[e] : o.Ve[e]) : (q == j ? o.D : o.V);
        }
        apply3(&v[(size_t)(n * 3 + k) * N3], N, M[0], Ms[0], M[1], Ms[1], M[2], Ms[2], A.data());
        for (int q = 0; q < 3; ++q) M[q] = q == d ? (q == k ? o.De[e] : o.Ve[e]) : (q == k ? o.D : o.V);
        apply3(&v[(size_t)(n * 3 + j) * N3], N, M[0], Ms[0], M[1], Ms[1], M[2], Ms[2], B.data());
        for (int r = 0; r < Nf; ++r) S_face[((size_t)f * 9 + i * 3 + n) * Nf + r] = -(A[r] - B[r]);
      }
  }
}

void prism18_curl(const CurvedOps &o, const TriBasis &tb, const double (*X)[3], double *S_sol, double *S_face) {
  const int N = o.N, Nt = tb.Nt, Np = Nt * N, Nf = N * N;
  std::vector<double> v;
  curl_fields(o.p, Np, 6, X, [&](int node, double x[3], double J[3][3]) {
    const double xi[3] = {tb.r[node % Nt], tb.s[node % Nt], o.g[node / Nt]};
    prism18_point(X, xi, x, J);
  }, v);
  // Triangle-part operators at the three kinds of targets: value / d/dr / d/ds.
  std::vector<double> I((size_t)Nt * Nt, 0.0);
  for (int q = 0; q < Nt; ++q) I[(size_t)q * Nt + q] = 1.0;
  const double *Tsol[3] = {I.data(), tb.Dr.data(), tb.Ds.data()};
  std::vector<double> Ed[3][3];   // edge e: value, d/dr, d/ds at its Gauss points [N][Nt]
  for (int e = 0; e < 3; ++e) {
    Ed[e][0] = tb.E[e];
    for (int w = 1; w < 3; ++w) {
      const std::vector<double> &Dm = w == 1 ? tb.Dr : tb.Ds;
      Ed[e][w].assign((size_t)N * Nt, 0.0);
      for (int a = 0; a < N; ++a)
        for (int q = 0; q < Nt; ++q) {
          double s = 0.0;
          for (int t = 0; t < Nt; ++t) s += tb.E[e][(size_t)a * Nt + t] * Dm[(size_t)t * Nt + q];
          Ed[e][w][(size_t)a * Nt + q] = s;
        }
    }
  }
  std::vector<double> A(Np), B(Np);
  // d/dxi_w of field F at targets (triangle operator set Tw, zeta value/derivative matrices).
  auto deriv = [&](const double *F, int w, const double *const *Tw, int T, const double *Zv, const double *Zd, int M,
                   double *out) {
    apply_tz(F, Nt, N, Tw[w < 2 ? w + 1 : 0], T, w == 2 ? Zd : Zv, M, out);
  };
  for (int n = 0; n < 3; ++n)
    for (int i = 0; i < 3; ++i) {
      const int j = (i + 1) % 3, k = (i + 2) % 3;
      deriv(&v[(size_t)(n * 3 + k) * Np], j, Tsol, Nt, o.V, o.D, N, A.data());
      deriv(&v[(size_t)(n * 3 + j) * Np], k, Tsol, Nt, o.V, o.D, N, B.data());
      for (int m = 0; m < Np; ++m) S_sol[(size_t)(i * 3 + n) * Np + m] = -(A[m] - B[m]);
      for (int f = 0; f < 2; ++f) {     // triangles at zeta = -1, +1
        deriv(&v[(size_t)(n * 3 + k) * Np], j, Tsol, Nt, o.Ve[f], o.De[f], 1, A.data());
        deriv(&v[(size_t)(n * 3 + j) * Np], k, Tsol, Nt, o.Ve[f], o.De[f], 1, B.data());
        for (int q = 0; q < Nt; ++q) S_face[((size_t)f * 9 + i * 3 + n) * Nf + q] = -(A[q] - B[q]);
      }
      for (int e = 0; e < 3; ++e) {     // quadrilaterals: edge Gauss points x zeta Gauss points
        const double *Te[3] = {Ed[e][0].data(), Ed[e][1].data(), Ed[e][2].data()};
        deriv(&v[(size_t)(n * 3 + k) * Np], j, Te, N, o.V, o.D, N, A.data());
        deriv(&v[(size_t)(n * 3 + j) * Np], k, Te, N, o.V, o.D, N, B.data());
        for (int r = 0; r < Nf; ++r) S_face[((size_t)(2 + e) * 9 + i * 3 + n) * Nf + r] = -(A[r] - B[r]);
      }
    }
}

}  // namespace frx
