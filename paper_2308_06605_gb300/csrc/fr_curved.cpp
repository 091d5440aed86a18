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
// coordinates small against the element.  Everything is evaluated one axis at a time: the
// quadratic map through 1D quadratic Lagrange matrices (the triangle's 6 quadratic functions on
// the prism), the interpolant's derivatives through 1D Lagrange matrices from the Gauss-Lobatto
// points and the triangle's nodal derivative and edge-interpolation matrices.
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
// Prism: (triangle function: 0..2 corners, 3..5 midpoints of 01 12 20; zeta level -1, 0, 1).
const int kPrism18[18][2] = {{0, -1}, {1, -1}, {2, -1}, {0, 1}, {1, 1}, {2, 1}, {3, -1}, {4, -1}, {5, -1},
                             {3, 1},  {4, 1},  {5, 1},  {0, 0}, {1, 0}, {2, 0}, {3, 0},  {4, 0},  {5, 0}};

// Quadratic Lagrange functions of the nodes -1, 0, 1 at t.
void quad3(double t, double L[3], double dL[3]) {
  L[0] = 0.5 * t * (t - 1.0); dL[0] = t - 0.5;
  L[1] = 1.0 - t * t;         dL[1] = -2.0 * t;
  L[2] = 0.5 * t * (t + 1.0); dL[2] = t + 0.5;
}

// The 6 quadratic triangle functions and their r, s derivatives at (r, s).
void tri6(double r, double s, double T[6], double Tr[6], double Ts[6]) {
  const double lam[3] = {-(r + s) / 2, (1 + r) / 2, (1 + s) / 2};
  const double dr[3] = {-0.5, 0.5, 0.0}, ds[3] = {-0.5, 0.0, 0.5};
  for (int i = 0; i < 3; ++i) {
    T[i] = lam[i] * (2 * lam[i] - 1);
    Tr[i] = (4 * lam[i] - 1) * dr[i];
    Ts[i] = (4 * lam[i] - 1) * ds[i];
  }
  const int mid[3][2] = {{0, 1}, {1, 2}, {2, 0}};
  for (int k = 0; k < 3; ++k) {
    const int i = mid[k][0], j = mid[k][1];
    T[3 + k] = 4 * lam[i] * lam[j];
    Tr[3 + k] = 4 * (dr[i] * lam[j] + lam[i] * dr[j]);
    Ts[3 + k] = 4 * (ds[i] * lam[j] + lam[i] * ds[j]);
  }
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

// out[i0 + M0 i1 + M0 M1 i2] = sum A0[i0][a] A1[i1][b] A2[i2][c] f[a + n b + n^2 c] (n inputs per axis).
void apply3(const double *f, int n, const double *A0, int M0, const double *A1, int M1, const double *A2, int M2,
            double *out, std::vector<double> &t1, std::vector<double> &t2) {
  t1.resize((size_t)M0 * n * n);
  t2.resize((size_t)M0 * M1 * n);
  for (int c = 0; c < n; ++c)
    for (int b = 0; b < n; ++b)
      for (int i = 0; i < M0; ++i) {
        double s = 0.0;
        for (int a = 0; a < n; ++a) s += A0[i * n + a] * f[a + n * b + n * n * c];
        t1[i + (size_t)M0 * (b + (size_t)n * c)] = s;
      }
  for (int c = 0; c < n; ++c)
    for (int j = 0; j < M1; ++j)
      for (int i = 0; i < M0; ++i) {
        double s = 0.0;
        for (int b = 0; b < n; ++b) s += A1[j * n + b] * t1[i + (size_t)M0 * (b + (size_t)n * c)];
        t2[i + (size_t)M0 * (j + (size_t)M1 * c)] = s;
      }
  for (int k = 0; k < M2; ++k)
    for (int j = 0; j < M1; ++j)
      for (int i = 0; i < M0; ++i) {
        double s = 0.0;
        for (int c = 0; c < n; ++c) s += A2[k * n + c] * t2[i + (size_t)M0 * (j + (size_t)M1 * c)];
        out[i + (size_t)M0 * (j + (size_t)M1 * k)] = s;
      }
}

// out[t + T z] = sum_q sum_k A[t][q] Z[z][k] f[q + nq k]  (triangle part, then zeta part).
void apply_tz(const double *f, int nq, int nk, const double *A, int T, const double *Z, int M, double *out,
              std::vector<double> &t1) {
  t1.resize((size_t)T * nk);
  for (int k = 0; k < nk; ++k)
    for (int t = 0; t < T; ++t) {
      double s = 0.0;
      for (int q = 0; q < nq; ++q) s += A[(size_t)t * nq + q] * f[q + (size_t)nq * k];
      t1[t + (size_t)T * k] = s;
    }
  for (int z = 0; z < M; ++z)
    for (int t = 0; t < T; ++t) {
      double s = 0.0;
      for (int k = 0; k < nk; ++k) s += Z[z * nk + k] * t1[t + (size_t)T * k];
      out[t + (size_t)T * z] = s;
    }
}

double det3(const double J[3][3]) {
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

// v[(n*3 + k)*nn + node] = (X_l - c_l) dX_m/dxi_k, (n, m, l) cyclic, from x [3][nn] and
// J [3 (component)][3 (direction)][nn] at the interpolation nodes.
void curl_fields(int p, int nn, int n_corner, const double (*X)[3], const double *x, const double *J,
                 std::vector<double> &v) {
  double c[3] = {0.0, 0.0, 0.0};
  if (p >= 2)
    for (int a = 0; a < n_corner; ++a)
      for (int i = 0; i < 3; ++i) c[i] += X[a][i] / n_corner;
  v.resize((size_t)9 * nn);
  for (int n = 0; n < 3; ++n) {
    const int m = (n + 1) % 3, l = (n + 2) % 3;
    for (int k = 0; k < 3; ++k)
      for (int node = 0; node < nn; ++node)
        v[(size_t)(n * 3 + k) * nn + node] = (x[(size_t)l * nn + node] - c[l]) * J[((size_t)m * 3 + k) * nn + node];
  }
}

}  // namespace

void curved_ops(int p, const Basis1D &b, const TriBasis *tb, CurvedOps &o) {
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
  for (int i = 0; i < N; ++i) {
    quad3(o.g[i], &o.Qg[i * 3], &o.dQg[i * 3]);
    quad3(b.x[i], &o.Qx[i * 3], &o.dQx[i * 3]);
  }
  quad3(-1.0, &o.Qe[0], &o.dQe[0]);
  quad3(1.0, &o.Qe[3], &o.dQe[3]);
  if (!tb) return;
  const int Nt = tb->Nt;
  o.Nt = Nt;
  o.T.resize((size_t)Nt * 6);
  o.Tr.resize((size_t)Nt * 6);
  o.Ts.resize((size_t)Nt * 6);
  for (int q = 0; q < Nt; ++q) tri6(tb->r[q], tb->s[q], &o.T[q * 6], &o.Tr[q * 6], &o.Ts[q * 6]);
  for (int e = 0; e < 3; ++e) {
    o.TE[e].resize((size_t)N * 6);
    o.TEr[e].resize((size_t)N * 6);
    o.TEs[e].resize((size_t)N * 6);
    for (int a = 0; a < N; ++a) {
      double r, s;
      tri_edge_point(e, b.x[a], r, s);
      tri6(r, s, &o.TE[e][a * 6], &o.TEr[e][a * 6], &o.TEs[e][a * 6]);
    }
  }
}

void hex27_geometry(const CurvedOps &o, const double (*X)[3], double *x_sol, double *det, double *S_sol,
                    double *x_face, double *S_face) {
  const int N = o.N, N3 = N * N * N, Nf = N * N;
  std::vector<double> t1, t2;
  // Node coordinates as 3 x 3 x 3 tensors per component.
  double Xt[3][27];
  for (int a = 0; a < 27; ++a)
    for (int c = 0; c < 3; ++c) Xt[c][(kHex27[a][0] + 1) + 3 * (kHex27[a][1] + 1) + 9 * (kHex27[a][2] + 1)] = X[a][c];
  // Position and gradient of the map at a tensor target set (1D value / derivative matrices).
  auto map_at = [&](const double *Q[3], const double *dQ[3], const int M[3], double *x, double *J) {
    const int nt = M[0] * M[1] * M[2];
    for (int c = 0; c < 3; ++c) {
      apply3(Xt[c], 3, Q[0], M[0], Q[1], M[1], Q[2], M[2], x + (size_t)c * nt, t1, t2);
      if (!J) continue;
      for (int d = 0; d < 3; ++d) {
        const double *A[3] = {Q[0], Q[1], Q[2]};
        A[d] = dQ[d];
        apply3(Xt[c], 3, A[0], M[0], A[1], M[1], A[2], M[2], J + ((size_t)c * 3 + d) * nt, t1, t2);
      }
    }
  };
  // Curl fields at the Gauss-Lobatto nodes.
  std::vector<double> xg((size_t)3 * N3), Jg((size_t)9 * N3), v;
  {
    const double *Q[3] = {o.Qg, o.Qg, o.Qg}, *dQ[3] = {o.dQg, o.dQg, o.dQg};
    const int M[3] = {N, N, N};
    map_at(Q, dQ, M, xg.data(), Jg.data());
  }
  curl_fields(o.p, N3, 8, X, xg.data(), Jg.data(), v);
  std::vector<double> A(N3), B(N3);
  // Row i of S at a tensor target set: axis d takes (value V, derivative D) matrices Vm[d], Dm[d].
  auto srow = [&](int i, const double *Vm[3], const double *Dm[3], const int M[3], double *out, size_t stride) {
    const int j = (i + 1) % 3, k = (i + 2) % 3, nt = M[0] * M[1] * M[2];
    for (int n = 0; n < 3; ++n) {
      const double *Aj[3] = {Vm[0], Vm[1], Vm[2]}, *Ak[3] = {Vm[0], Vm[1], Vm[2]};
      Aj[j] = Dm[j];
      Ak[k] = Dm[k];
      apply3(&v[(size_t)(n * 3 + k) * N3], N, Aj[0], M[0], Aj[1], M[1], Aj[2], M[2], A.data(), t1, t2);
      apply3(&v[(size_t)(n * 3 + j) * N3], N, Ak[0], M[0], Ak[1], M[1], Ak[2], M[2], B.data(), t1, t2);
      for (int r = 0; r < nt; ++r) out[(size_t)(i * 3 + n) * stride + r] = -(A[r] - B[r]);
    }
  };
  // Solution points: position, |J| and all of S.
  {
    const double *Q[3] = {o.Qx, o.Qx, o.Qx}, *dQ[3] = {o.dQx, o.dQx, o.dQx};
    const int M[3] = {N, N, N};
    std::vector<double> xs((size_t)3 * N3), Js((size_t)9 * N3);
    map_at(Q, dQ, M, xs.data(), Js.data());
    for (int m = 0; m < N3; ++m) {
      double J[3][3];
      for (int c = 0; c < 3; ++c) {
        x_sol[(size_t)m * 3 + c] = xs[(size_t)c * N3 + m];
        for (int d = 0; d < 3; ++d) J[c][d] = Js[((size_t)c * 3 + d) * N3 + m];
      }
      det[m] = det3(J);
    }
    const double *Vm[3] = {o.V, o.V, o.V}, *Dm[3] = {o.D, o.D, o.D};
    for (int i = 0; i < 3; ++i) srow(i, Vm, Dm, M, S_sol, N3);
  }
  // Faces: axis d at its end e, the tangential axes on the Gauss-Legendre points; the flux point
  // r = a + N b runs over the two tangential axes in increasing order, so it is the tensor index.
  for (int f = 0; f < 6; ++f) {
    const int d = f / 2, e = f % 2;
    const double *Q[3] = {o.Qx, o.Qx, o.Qx}, *Vm[3] = {o.V, o.V, o.V}, *Dm[3] = {o.D, o.D, o.D};
    Q[d] = &o.Qe[3 * e];
    Vm[d] = o.Ve[e];
    Dm[d] = o.De[e];
    int M[3] = {N, N, N};
    M[d] = 1;
    std::vector<double> xf((size_t)3 * Nf);
    map_at(Q, nullptr, M, xf.data(), nullptr);
    for (int r = 0; r < Nf; ++r)
      for (int c = 0; c < 3; ++c) x_face[((size_t)f * Nf + r) * 3 + c] = xf[(size_t)c * Nf + r];
    srow(d, Vm, Dm, M, S_face + (size_t)f * 9 * Nf, Nf);
  }
}

void prism18_geometry(const CurvedOps &o, const TriBasis &tb, const double (*X)[3], double *x_sol, double *det,
                      double *S_sol, double *x_face, double *S_face) {
  const int N = o.N, Nt = tb.Nt, Np = Nt * N, Nf = N * N;
  std::vector<double> t1;
  double Xt[3][18];   // [component][triangle function + 6 level]
  for (int a = 0; a < 18; ++a)
    for (int c = 0; c < 3; ++c) Xt[c][kPrism18[a][0] + 6 * (kPrism18[a][1] + 1)] = X[a][c];
  // Map at (triangle targets via T/Tr/Ts [T][6]) x (zeta targets via Z/dZ [M][3]).
  auto map_at = [&](const double *Tv, const double *Trm, const double *Tsm, int T, const double *Z, const double *dZ,
                    int M, double *x, double *J) {
    const int nt = T * M;
    for (int c = 0; c < 3; ++c) {
      apply_tz(Xt[c], 6, 3, Tv, T, Z, M, x + (size_t)c * nt, t1);
      if (!J) continue;
      apply_tz(Xt[c], 6, 3, Trm, T, Z, M, J + ((size_t)c * 3 + 0) * nt, t1);
      apply_tz(Xt[c], 6, 3, Tsm, T, Z, M, J + ((size_t)c * 3 + 1) * nt, t1);
      apply_tz(Xt[c], 6, 3, Tv, T, dZ, M, J + ((size_t)c * 3 + 2) * nt, t1);
    }
  };
  std::vector<double> xg((size_t)3 * Np), Jg((size_t)9 * Np), v;
  map_at(o.T.data(), o.Tr.data(), o.Ts.data(), Nt, o.Qg, o.dQg, N, xg.data(), Jg.data());
  curl_fields(o.p, Np, 6, X, xg.data(), Jg.data(), v);
  // Triangle-part operators: value / d/dr / d/ds at the nodes and at each edge's Gauss points.
  std::vector<double> I((size_t)Nt * Nt, 0.0);
  for (int q = 0; q < Nt; ++q) I[(size_t)q * Nt + q] = 1.0;
  const double *Tn[3] = {I.data(), tb.Dr.data(), tb.Ds.data()};
  std::vector<double> Ed[3][3];
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
  // d/dxi_w of a field at targets (triangle operators Tw[value, r, s], zeta value/derivative).
  auto deriv = [&](const double *F, int w, const double *const *Tw, int T, const double *Zv, const double *Zd, int M,
                   double *out) { apply_tz(F, Nt, N, Tw[w < 2 ? w + 1 : 0], T, w == 2 ? Zd : Zv, M, out, t1); };
  auto srow = [&](int i, const double *const *Tw, int T, const double *Zv, const double *Zd, int M, double *out,
                  size_t stride) {
    const int j = (i + 1) % 3, k = (i + 2) % 3;
    for (int n = 0; n < 3; ++n) {
      deriv(&v[(size_t)(n * 3 + k) * Np], j, Tw, T, Zv, Zd, M, A.data());
      deriv(&v[(size_t)(n * 3 + j) * Np], k, Tw, T, Zv, Zd, M, B.data());
      for (int r = 0; r < T * M; ++r) out[(size_t)(i * 3 + n) * stride + r] = -(A[r] - B[r]);
    }
  };
  {
    std::vector<double> xs((size_t)3 * Np), Js((size_t)9 * Np);
    map_at(o.T.data(), o.Tr.data(), o.Ts.data(), Nt, o.Qx, o.dQx, N, xs.data(), Js.data());
    for (int m = 0; m < Np; ++m) {
      double J[3][3];
      for (int c = 0; c < 3; ++c) {
        x_sol[(size_t)m * 3 + c] = xs[(size_t)c * Np + m];
        for (int d = 0; d < 3; ++d) J[c][d] = Js[((size_t)c * 3 + d) * Np + m];
      }
      det[m] = det3(J);
    }
    for (int i = 0; i < 3; ++i) srow(i, Tn, Nt, o.V, o.D, N, S_sol, Np);
  }
  std::vector<double> xf((size_t)3 * Nf);
  for (int f = 0; f < 2; ++f) {            // triangles at zeta = -1, +1: row 2 of S
    map_at(o.T.data(), nullptr, nullptr, Nt, &o.Qe[3 * f], nullptr, 1, xf.data(), nullptr);
    for (int r = 0; r < Nt; ++r)
      for (int c = 0; c < 3; ++c) x_face[((size_t)f * Nf + r) * 3 + c] = xf[(size_t)c * Nt + r];
    srow(2, Tn, Nt, o.Ve[f], o.De[f], 1, S_face + (size_t)f * 9 * Nf, Nf);
  }
  for (int e = 0; e < 3; ++e) {            // quadrilaterals (edge Gauss points x zeta Gauss points): rows 0, 1
    map_at(o.TE[e].data(), nullptr, nullptr, N, o.Qx, nullptr, N, xf.data(), nullptr);
    for (int r = 0; r < Nf; ++r)
      for (int c = 0; c < 3; ++c) x_face[((size_t)(2 + e) * Nf + r) * 3 + c] = xf[(size_t)c * Nf + r];
    const double *Te[3] = {Ed[e][0].data(), Ed[e][1].data(), Ed[e][2].data()};
    for (int i = 0; i < 2; ++i) srow(i, Te, N, o.V, o.D, N, S_face + (size_t)(2 + e) * 9 * Nf, Nf);
  }
}

}  // namespace frx
