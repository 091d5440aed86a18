// Host-side construction of the FR discretisation: 1D basis, face connectivity, orientation
// codes and element metrics (arXiv 2308.06605, section "FR Algorithm", Eq. 1-2, and the face
// construction of the pre-processor section: faces keyed by sorted vertex ids, sorted so that
// coupled faces are adjacent, then paired).
#include <algorithm>
#include <array>
#include <atomic>
#include <climits>
#include <thread>
#include <cmath>
#include <cstdio>
#include <unordered_map>

#include "fr_internal.hpp"

namespace frx {

using ld = long double;

// ------------------------------------------------------------------------------------------
// Gauss-Legendre nodes by Golub-Welsch: eigenvalues of the symmetric tridiagonal Jacobi matrix
// of the Legendre recurrence (zero diagonal, off-diagonal k / sqrt(4k^2 - 1)), found with the
// implicit QL iteration, then polished by Newton steps on P_N.
// ------------------------------------------------------------------------------------------
static void tridiag_ql(int n, ld *d, ld *e) {
  for (int l = 0; l < n; ++l) {
    for (int iter = 0; iter < 200; ++iter) {
      int m = l;
      for (; m < n - 1; ++m) {
        ld dd = fabsl(d[m]) + fabsl(d[m + 1]);
        if (fabsl(e[m]) <= 1e-30L * dd + 1e-300L) break;
      }
      if (m == l) break;
      ld g = (d[l + 1] - d[l]) / (2.0L * e[l]);
      ld r = sqrtl(g * g + 1.0L);
      g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
      ld s = 1.0L, c = 1.0L, p = 0.0L;
      int i = m - 1;
      bool underflow = false;
      for (; i >= l; --i) {
        ld f = s * e[i], b = c * e[i];
        r = sqrtl(f * f + g * g);
        e[i + 1] = r;
        if (r == 0.0L) { d[i + 1] -= p; e[m] = 0.0L; underflow = true; break; }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0L * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
      }
      if (underflow) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0L;
    }
  }
}

static void legendre_pd(int n, ld x, ld &P, ld &dP) {
  ld p0 = 1.0L, p1 = x;
  if (n == 0) { P = 1.0L; dP = 0.0L; return; }
  for (int k = 1; k < n; ++k) {
    ld p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    p0 = p1;
    p1 = p2;
  }
  P = p1;
  dP = n * (p0 - x * p1) / (1.0L - x * x);   // valid inside (-1, 1)
}

// eta_p = c (2p + 1) (a_p p!)^2 / 2 of the energy-stable family, a_p p! = (2p)! / (2^p p!) the
// leading coefficient of P_p times p!.
static ld vcjh_eta(int p, double c) {
  ld apf = 1.0L;
  for (int k = p + 1; k <= 2 * p; ++k) apf *= (ld)k;   // (2p)! / p!
  for (int k = 0; k < p; ++k) apf *= 0.5L;
  return (ld)c * (2 * p + 1) * apf * apf / 2;
}

Basis1D make_basis(int p, double c) {
  Basis1D b;
  const int N = p + 1;
  b.p = p;
  b.N = N;
  ld d[kMaxN] = {0}, e[kMaxN] = {0}, x[kMaxN], w[kMaxN];
  for (int k = 1; k < N; ++k) e[k - 1] = (ld)k / sqrtl(4.0L * k * k - 1.0L);
  tridiag_ql(N, d, e);
  std::sort(d, d + N);
  for (int i = 0; i < N; ++i) {
    ld xi = d[i];
    for (int it = 0; it < 3; ++it) {
      ld P, dP;
      legendre_pd(N, xi, P, dP);
      xi -= P / dP;
    }
    x[i] = xi;
  }
  for (int i = 0; i < N / 2; ++i) {            // exact symmetry x_{N-1-i} = -x_i
    ld s = 0.5L * (x[N - 1 - i] - x[i]);
    x[i] = -s;
    x[N - 1 - i] = s;
  }
  if (N % 2) x[N / 2] = 0.0L;
  for (int i = 0; i < N; ++i) {
    ld P, dP;
    legendre_pd(N, x[i], P, dP);
    w[i] = 2.0L / ((1.0L - x[i] * x[i]) * dP * dP);
  }
  // Barycentric weights, derivative matrix and boundary values of the Lagrange basis.
  ld lam[kMaxN];
  for (int j = 0; j < N; ++j) {
    ld q = 1.0L;
    for (int m = 0; m < N; ++m)
      if (m != j) q *= (x[j] - x[m]);
    lam[j] = 1.0L / q;
  }
  for (int i = 0; i < N; ++i) {
    ld diag = 0.0L;
    for (int j = 0; j < N; ++j) {
      if (j == i) continue;
      ld v = (lam[j] / lam[i]) / (x[i] - x[j]);
      b.D[i * N + j] = (double)v;
      diag -= v;
    }
    b.D[i * N + i] = (double)diag;
  }
  for (int side = 0; side < 2; ++side) {
    ld xe = side ? 1.0L : -1.0L, den = 0.0L;
    for (int k = 0; k < N; ++k) den += lam[k] / (xe - x[k]);
    for (int j = 0; j < N; ++j) {
      ld v = (lam[j] / (xe - x[j])) / den;
      if (side) b.lp[j] = (double)v; else b.lm[j] = (double)v;
    }
  }
  // DG-equivalent (c = 0) correction: on Gauss-Legendre points the derivative of the right
  // Radau polynomial equals the lifting l_i(1) / w_i (exact mass matrix), and by symmetry the
  // left one's (negated, mirrored) equals l_i(-1) / w_i.
  for (int i = 0; i < N; ++i) {
    b.x[i] = (double)x[i];
    b.w[i] = (double)w[i];
    ld lpv = 0, lmv = 0;
    {
      ld den = 0.0L;
      for (int k = 0; k < N; ++k) den += lam[k] / (1.0L - x[k]);
      lpv = (lam[i] / (1.0L - x[i])) / den;
      den = 0.0L;
      for (int k = 0; k < N; ++k) den += lam[k] / (-1.0L - x[k]);
      lmv = (lam[i] / (-1.0L - x[i])) / den;
    }
    b.hp[i] = (double)(lpv / w[i]);
    b.hm[i] = (double)(lmv / w[i]);
  }
  // Energy-stable family (Vincent, Castonguay & Jameson 2011): relative to the Radau member the
  // right correction changes by eta/(2(1+eta)) (P_{p-1} - P_{p+1}), whose derivative is
  // -kappa P_p with kappa = (2p+1) eta / (2 (1 + eta)) (Legendre: P'_{p+1} - P'_{p-1} = (2p+1) P_p).
  // hp = g_R'(x_i) and hm = g_R'(-x_i) = -g_L'(x_i), P_p(-x) = (-1)^p P_p(x).
  if (c != 0.0) {
    const ld eta = vcjh_eta(p, c), kap = (2 * p + 1) * eta / (2 * (1 + eta));
    for (int i = 0; i < N; ++i) {
      ld P, dP;
      legendre_pd(p, x[i], P, dP);
      b.hp[i] = (double)((ld)b.hp[i] - kap * P);
      b.hm[i] = (double)((ld)b.hm[i] - kap * ((p % 2) ? -P : P));
    }
  }
  return b;
}

bool vcjh_in_family(int p, double c) {
  if (!std::isfinite(c)) return false;
  const ld eta = vcjh_eta(p, c);
  return std::isfinite((double)eta) && 1 + eta > 0;
}

}  // namespace frx

extern "C" fr_status fr_basis_1d(int32_t p, double c, double *x, double *w, double *D, double *lm, double *lp,
                                 double *hm, double *hp) {
  if (p < 1 || p > 7 || !frx::vcjh_in_family(p, c)) return FR_EINVAL;
  const frx::Basis1D b = frx::make_basis(p, c);
  const int N = p + 1;
  for (int i = 0; i < N; ++i) {
    if (x) x[i] = b.x[i];
    if (w) w[i] = b.w[i];
    if (lm) lm[i] = b.lm[i];
    if (lp) lp[i] = b.lp[i];
    if (hm) hm[i] = b.hm[i];
    if (hp) hp[i] = b.hp[i];
    for (int a = 0; a < N; ++a)
      if (D) D[i * N + a] = b.D[i * N + a];
  }
  return FR_OK;
}

namespace frx {

// ------------------------------------------------------------------------------------------
// Geometry of the trilinear hexahedron.
// ------------------------------------------------------------------------------------------
static const int kVert[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};

struct Jac {
  double x[3];
  double J[3][3];   // J[i][b] = dx_i / dxi_b
};

static Jac trilinear(const double (*X)[3], const double xi[3]) {
  Jac r{};
  for (int v = 0; v < 8; ++v) {
    double f[3];
    for (int a = 0; a < 3; ++a) f[a] = 0.5 * (1.0 + kVert[v][a] * xi[a]);
    double Nv = f[0] * f[1] * f[2];
    double dN[3] = {0.5 * kVert[v][0] * f[1] * f[2], 0.5 * kVert[v][1] * f[0] * f[2],
                    0.5 * kVert[v][2] * f[0] * f[1]};
    for (int i = 0; i < 3; ++i) {
      r.x[i] += Nv * X[v][i];
      for (int b = 0; b < 3; ++b) r.J[i][b] += dN[b] * X[v][i];
    }
  }
  return r;
}

// S = |J| J^-1: row d is the cross product of the other two columns of J (cyclic order).
static void adjugate_rows(const double J[3][3], double S[3][3], double &det) {
  for (int d = 0; d < 3; ++d) {
    int b1 = (d + 1) % 3, b2 = (d + 2) % 3;
    S[d][0] = J[1][b1] * J[2][b2] - J[2][b1] * J[1][b2];
    S[d][1] = J[2][b1] * J[0][b2] - J[0][b1] * J[2][b2];
    S[d][2] = J[0][b1] * J[1][b2] - J[1][b1] * J[0][b2];
  }
  det = J[0][0] * S[0][0] + J[1][0] * S[0][1] + J[2][0] * S[0][2];
}

static inline void face_axes(int f, int &d, int &s, int &t0, int &t1) {
  d = f / 2;
  s = (f % 2) ? 1 : -1;
  t0 = (d == 0) ? 1 : 0;
  t1 = (d == 2) ? 1 : 2;
}

// ------------------------------------------------------------------------------------------
// Connectivity.
// ------------------------------------------------------------------------------------------
struct FaceRec {
  std::array<int64_t, 4> key;
  int64_t e;
  int f;
};

struct Side {
  int64_t e;
  int f;
};

static void face_corners(const int64_t *hex, int stride, int64_t e, int f, int64_t out[4], int ref[4][2]) {
  int d, s, t0, t1;
  face_axes(f, d, s, t0, t1);
  int c = 0;
  for (int v = 0; v < 8; ++v) {
    if (kVert[v][d] != s) continue;
    out[c] = hex[e * stride + v];
    ref[c][0] = kVert[v][t0];
    ref[c][1] = kVert[v][t1];
    ++c;
  }
}

// Orientation code mapping side-1 face coordinates onto side-0 face coordinates.
static int find_orientation(const double c0[4][3], const int r0[4][2], const double c1[4][3],
                            const int r1[4][2], const double shift1[3], double tol) {
  // For each side-1 corner find the side-0 corner at the same physical location.
  int match[4];
  for (int a = 0; a < 4; ++a) {
    match[a] = -1;
    for (int b = 0; b < 4; ++b) {
      double dx = c1[a][0] - shift1[0] - c0[b][0], dy = c1[a][1] - shift1[1] - c0[b][1],
             dz = c1[a][2] - shift1[2] - c0[b][2];
      if (dx * dx + dy * dy + dz * dz <= tol * tol) { match[a] = b; break; }
    }
    if (match[a] < 0) return -1;
  }
  for (int code = 0; code < 8; ++code) {
    bool ok = true;
    for (int a = 0; a < 4 && ok; ++a) {
      int u = r1[a][0], v = r1[a][1];
      if (code & 4) std::swap(u, v);
      if (code & 1) u = -u;
      if (code & 2) v = -v;
      ok = (u == r0[match[a]][0] && v == r0[match[a]][1]);
    }
    if (ok) return code;
  }
  return -1;
}

// Triangular faces: the vertex permutation (kTriPerm code) carrying side-1 corners onto the
// side-0 corners at the same physical location.
static int find_tri_orientation(const double c0[4][3], const double c1[4][3], const double shift1[3], double tol) {
  int match[3];
  for (int a = 0; a < 3; ++a) {
    match[a] = -1;
    for (int b = 0; b < 3; ++b) {
      double dx = c1[a][0] - shift1[0] - c0[b][0], dy = c1[a][1] - shift1[1] - c0[b][1],
             dz = c1[a][2] - shift1[2] - c0[b][2];
      if (dx * dx + dy * dy + dz * dz <= tol * tol) { match[a] = b; break; }
    }
    if (match[a] < 0) return -1;
  }
  for (int c = 0; c < 6; ++c)
    if (kTriPerm[c][0] == match[0] && kTriPerm[c][1] == match[1] && kTriPerm[c][2] == match[2]) return c;
  return -1;
}

// ------------------------------------------------------------------------------------------
// Geometry of the 6-node prism: vertices (-1,-1,-1), (1,-1,-1), (-1,1,-1) and the same at
// zeta = +1 (VTK wedge order); linear on the triangle times linear in zeta.
// ------------------------------------------------------------------------------------------
static Jac prism_map(const double (*X)[3], const double xi[3]) {
  Jac g{};
  const double r = xi[0], s = xi[1], z = xi[2];
  const double lam[3] = {-(r + s) / 2, (1 + r) / 2, (1 + s) / 2};
  const double dlr[3] = {-0.5, 0.5, 0.0}, dls[3] = {-0.5, 0.0, 0.5};
  const double lo = (1 - z) / 2, hi = (1 + z) / 2;
  for (int v = 0; v < 6; ++v) {
    const int t = v % 3;
    const double wz = v < 3 ? lo : hi, dz = v < 3 ? -0.5 : 0.5;
    const double Nv = lam[t] * wz;
    const double dN[3] = {dlr[t] * wz, dls[t] * wz, lam[t] * dz};
    for (int i = 0; i < 3; ++i) {
      g.x[i] += Nv * X[v][i];
      for (int b = 0; b < 3; ++b) g.J[i][b] += dN[b] * X[v][i];
    }
  }
  return g;
}

// Prism faces: 0 zeta = -1, 1 zeta = +1 (triangles; corners with reference (r, s) below), 2 s = -1,
// 3 r + s = 0, 4 r = -1 (quadrilaterals; corners with (sigma, zeta) coordinates below, sigma the
// parameter of triangle edge f - 2).
static const int kPrismFace[5][4] = {{0, 1, 2, -1}, {3, 4, 5, -1}, {0, 1, 4, 3}, {1, 2, 5, 4}, {2, 0, 3, 5}};
static const int kTriRef[3][2] = {{-1, -1}, {1, -1}, {-1, 1}};
static const int kQuadRef[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
// Reference normal of prism face f, scaled by the face's measure per unit parameter area.
static const double kPrismNormal[5][3] = {{0, 0, -1}, {0, 0, 1}, {0, -1, 0}, {1, 1, 0}, {-1, 0, 0}};

struct FaceGeo {
  int nc;                // corners: 4 quadrilateral, 3 triangle
  int64_t ids[4];
  int ref[4][2];
};

// Runs body(begin, end) over [0, n) split across host threads (serially for small n).
template <typename F>
static void parallel_for(int64_t n, F body) {
  unsigned nt = std::thread::hardware_concurrency();
  nt = nt == 0 ? 1 : (nt > 32 ? 32 : nt);
  if (n < 512 || nt <= 1) {
    body(0, n);
    return;
  }
  std::vector<std::thread> th;
  const int64_t chunk = (n + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    const int64_t b = (int64_t)t * chunk, e = std::min<int64_t>(n, b + chunk);
    if (b < e) th.emplace_back(body, b, e);
  }
  for (std::thread &x : th) x.join();
}

fr_status build_host_mesh(const fr_mesh_desc *desc, HostMesh &m, std::string &err, double vcjh_c) {
  char buf[256];
  const int p = desc->p;
  const int N = p + 1, Np = N * N * N, Nf = N * N;
  const int64_t E = desc->n_hex;
  const int64_t Ep = desc->n_prism > 0 ? desc->n_prism : 0;
  const int64_t G = E + Ep;                 // elements: hexahedra first, then prisms
  const int hn = desc->hex_nodes == 0 ? 8 : desc->hex_nodes, pn = desc->prism_nodes == 0 ? 6 : desc->prism_nodes;
  if ((hn != 8 && hn != 27) || (pn != 6 && pn != 18)) {
    err = "hex_nodes must be 8 or 27 and prism_nodes 6 or 18";
    return FR_EINVAL;
  }
  m.p = p; m.N = N; m.Np = Np; m.Nf = Nf; m.E = E; m.Ep = Ep;
  for (int64_t i = 0; i < E * hn; ++i) {
    if (desc->hex[i] < 0 || desc->hex[i] >= desc->n_nodes) {
      err = "hex vertex id out of range";
      return FR_EINVAL;
    }
  }
  for (int64_t i = 0; i < Ep * pn; ++i) {
    if (desc->prism[i] < 0 || desc->prism[i] >= desc->n_nodes) {
      err = "prism vertex id out of range";
      return FR_EINVAL;
    }
  }
  if (G >= (int64_t(1) << 31)) {
    err = "too many elements for this build";
    return FR_EUNSUPPORTED;
  }
  TriBasis tb;
  if (Ep > 0) {
    if (!make_tri_basis(p, tb)) {
      err = "internal: triangle basis construction failed";
      return FR_EMESH;
    }
    m.Nt = tb.Nt;
    m.Npp = tb.Nt * N;
  }
  const int Nt = m.Nt, Npp = m.Npp;
  const double(*xyz)[3] = reinterpret_cast<const double(*)[3]>(desc->xyz);
  // Element nodes (the corners come first in both node orders).
  auto elem_verts = [&](int64_t e, double X[][3], int n = 8) {
    for (int v = 0; v < n; ++v)
      for (int i = 0; i < 3; ++i) X[v][i] = xyz[desc->hex[e * hn + v]][i];
  };
  auto prism_verts = [&](int64_t ep, double X[][3], int n = 6) {
    for (int v = 0; v < n; ++v)
      for (int i = 0; i < 3; ++i) X[v][i] = xyz[desc->prism[ep * pn + v]][i];
  };
  auto nfaces = [&](int64_t g) { return g < E ? 6 : 5; };
  auto face_index = [&](int64_t g, int f) { return g < E ? g * 6 + f : E * 6 + (g - E) * 5 + f; };
  auto face_geo = [&](int64_t g, int f, FaceGeo &F) {
    if (g < E) {
      F.nc = 4;
      face_corners(desc->hex, hn, g, f, F.ids, F.ref);
      return;
    }
    const int64_t *pv = desc->prism + (g - E) * pn;
    F.nc = f < 2 ? 3 : 4;
    for (int a = 0; a < F.nc; ++a) {
      F.ids[a] = pv[kPrismFace[f][a]];
      F.ref[a][0] = f < 2 ? kTriRef[a][0] : kQuadRef[a][0];
      F.ref[a][1] = f < 2 ? kTriRef[a][1] : kQuadRef[a][1];
    }
    if (F.nc == 3) {
      F.ids[3] = -1;
      F.ref[3][0] = F.ref[3][1] = 0;
    }
  };
  // Minimum element size for tolerances.
  double hmin = 1e300;
  for (int64_t e = 0; e < E; ++e) {
    double X[8][3];
    elem_verts(e, X);
    double dx = X[6][0] - X[0][0], dy = X[6][1] - X[0][1], dz = X[6][2] - X[0][2];
    hmin = std::min(hmin, std::sqrt(dx * dx + dy * dy + dz * dz));
  }
  for (int64_t ep = 0; ep < Ep; ++ep) {
    double X[6][3];
    prism_verts(ep, X);
    double dx = X[4][0] - X[0][0], dy = X[4][1] - X[0][1], dz = X[4][2] - X[0][2];
    hmin = std::min(hmin, std::sqrt(dx * dx + dy * dy + dz * dz));
  }
  const double tol = 1e-7 * hmin;

  // Faces keyed by sorted vertex ids (a triangle's key carries -1 in the fourth place); sorting
  // makes coupled faces adjacent.
  std::vector<FaceRec> faces((size_t)(E * 6 + Ep * 5));
  for (int64_t g = 0; g < G; ++g)
    for (int f = 0; f < nfaces(g); ++f) {
      FaceGeo F;
      face_geo(g, f, F);
      std::array<int64_t, 4> k = {F.ids[0], F.ids[1], F.ids[2], F.nc == 4 ? F.ids[3] : -1};
      std::sort(k.begin(), k.end());
      faces[face_index(g, f)] = {k, g, f};
    }
  std::sort(faces.begin(), faces.end(), [](const FaceRec &a, const FaceRec &b) {
    if (a.key != b.key) return a.key < b.key;
    return a.e * 6 + a.f < b.e * 6 + b.f;
  });
  std::vector<std::pair<Side, Side>> pairs;
  std::vector<FaceRec> open;
  for (size_t i = 0; i < faces.size();) {
    size_t j = i + 1;
    while (j < faces.size() && faces[j].key == faces[i].key) ++j;
    if (j - i == 2) {
      pairs.push_back({{faces[i].e, faces[i].f}, {faces[i + 1].e, faces[i + 1].f}});
    } else if (j - i == 1) {
      open.push_back(faces[i]);
    } else {
      snprintf(buf, sizeof buf, "face shared by %zu elements", j - i);
      err = buf;
      return FR_EMESH;
    }
    i = j;
  }
  // Boundary tags of the unpaired faces (a triangle lists -1 as its fourth vertex).
  std::vector<std::pair<std::array<int64_t, 4>, int32_t>> btags(desc->n_bface);
  for (int64_t i = 0; i < desc->n_bface; ++i) {
    std::array<int64_t, 4> k = {desc->bface_nodes[4 * i], desc->bface_nodes[4 * i + 1],
                                desc->bface_nodes[4 * i + 2], desc->bface_nodes[4 * i + 3]};
    std::sort(k.begin(), k.end());
    btags[i] = {k, desc->bface_tag[i]};
  }
  std::sort(btags.begin(), btags.end());
  struct Open { Side s; int32_t tag; double cent[3]; };
  std::vector<Open> opens;
  opens.reserve(open.size());
  for (const FaceRec &fr : open) {
    auto it = std::lower_bound(btags.begin(), btags.end(), std::make_pair(fr.key, INT32_MIN));
    if (it == btags.end() || it->first != fr.key) {
      err = "unmatched face with no boundary tag";
      return FR_EMESH;
    }
    Open o{{fr.e, fr.f}, it->second, {0, 0, 0}};
    int nc = 0;
    for (int c = 0; c < 4; ++c) nc += fr.key[c] >= 0;
    for (int c = 0; c < 4; ++c)
      if (fr.key[c] >= 0)
        for (int i = 0; i < 3; ++i) o.cent[i] += xyz[fr.key[c]][i] / nc;
    opens.push_back(o);
  }
  // Periodic pairing by translated centroids on a hashed grid.
  std::vector<int> used(opens.size(), 0);
  std::vector<std::array<double, 3>> pshift;   // shift of side 1 per periodic pair
  std::vector<std::pair<Side, Side>> ppairs;
  const double cell = 0.25 * hmin;
  for (int ip = 0; ip < desc->n_periodic; ++ip) {
    const fr_periodic &P = desc->periodic[ip];
    std::unordered_map<int64_t, std::vector<int>> grid;
    auto key_of = [&](const double c[3], int dx, int dy, int dz) {
      int64_t ix = (int64_t)std::floor(c[0] / cell) + dx, iy = (int64_t)std::floor(c[1] / cell) + dy,
              iz = (int64_t)std::floor(c[2] / cell) + dz;
      return (ix * 73856093LL) ^ (iy * 19349663LL) ^ (iz * 83492791LL);
    };
    for (size_t i = 0; i < opens.size(); ++i)
      if (opens[i].tag == P.tag_a) grid[key_of(opens[i].cent, 0, 0, 0)].push_back((int)i);
    for (size_t i = 0; i < opens.size(); ++i) {
      if (opens[i].tag != P.tag_b) continue;
      double c[3] = {opens[i].cent[0] - P.t[0], opens[i].cent[1] - P.t[1], opens[i].cent[2] - P.t[2]};
      int found = -1;
      for (int dx = -1; dx <= 1 && found < 0; ++dx)
        for (int dy = -1; dy <= 1 && found < 0; ++dy)
          for (int dz = -1; dz <= 1 && found < 0; ++dz) {
            auto it = grid.find(key_of(c, dx, dy, dz));
            if (it == grid.end()) continue;
            for (int j : it->second) {
              double ex = opens[j].cent[0] - c[0], ey = opens[j].cent[1] - c[1], ez = opens[j].cent[2] - c[2];
              if (!used[j] && ex * ex + ey * ey + ez * ez <= tol * tol) { found = j; break; }
            }
          }
      if (found < 0) {
        snprintf(buf, sizeof buf, "periodic face (tag %d) without a partner (tag %d)", P.tag_b, P.tag_a);
        err = buf;
        return FR_EMESH;
      }
      used[found] = 1;
      used[i] = 1;
      ppairs.push_back({opens[found].s, opens[i].s});
      pshift.push_back({P.t[0], P.t[1], P.t[2]});
    }
  }
  // Remaining open faces need a boundary condition.
  std::vector<std::pair<Side, int>> bfaces;
  m.bcs.clear();
  for (size_t i = 0; i < opens.size(); ++i) {
    if (used[i]) continue;
    int bi = -1;
    for (int k = 0; k < desc->n_bc; ++k)
      if (desc->bc[k].tag == opens[i].tag) bi = k;
    bool periodic_tag = false;
    for (int ip = 0; ip < desc->n_periodic; ++ip)
      periodic_tag |= (desc->periodic[ip].tag_a == opens[i].tag || desc->periodic[ip].tag_b == opens[i].tag);
    if (bi < 0 || periodic_tag) {
      snprintf(buf, sizeof buf, "boundary face with tag %d has no condition or partner", opens[i].tag);
      err = buf;
      return FR_EMESH;
    }
    bfaces.push_back({opens[i].s, bi});
  }
  if (desc->n_bc > kMaxBC) {
    err = "too many boundary conditions";
    return FR_EUNSUPPORTED;
  }
  for (int k = 0; k < desc->n_bc; ++k) m.bcs.push_back(desc->bc[k]);

  const int64_t n_int = (int64_t)pairs.size() + (int64_t)ppairs.size();
  m.n_interior = n_int;
  m.n_if = n_int + (int64_t)bfaces.size();
  if (m.n_if >= (int64_t(1) << 27)) {
    err = "too many interfaces for this build";
    return FR_EUNSUPPORTED;
  }
  m.ef.assign(E * 6, -1);
  m.ef_p.assign(Ep * 5, -1);
  m.if_bc.assign(m.n_if, -1);
  m.if_elem.assign(2 * m.n_if, -1);
  if (Ep > 0) m.if_tri.assign(m.n_if, 0);
  auto set_ef = [&](Side s, int32_t packed) {
    if (s.e < E) m.ef[s.e * 6 + s.f] = packed;
    else m.ef_p[(s.e - E) * 5 + s.f] = packed;
  };
  std::vector<int> orient(n_int, 0);
  // Orientation of side 1 relative to side 0.
  auto corner_xyz = [&](Side s, double c[4][3], FaceGeo &F) {
    face_geo(s.e, s.f, F);
    for (int k = 0; k < F.nc; ++k)
      for (int i = 0; i < 3; ++i) c[k][i] = xyz[F.ids[k]][i];
  };
  for (int64_t I = 0; I < n_int; ++I) {
    bool per = I >= (int64_t)pairs.size();
    const auto &pr = per ? ppairs[I - pairs.size()] : pairs[I];
    double shift[3] = {0, 0, 0};
    if (per)
      for (int i = 0; i < 3; ++i) shift[i] = pshift[I - pairs.size()][i];
    double c0[4][3], c1[4][3];
    FaceGeo F0, F1;
    corner_xyz(pr.first, c0, F0);
    corner_xyz(pr.second, c1, F1);
    if (F0.nc != F1.nc) {
      err = "a triangular face is paired with a quadrilateral";
      return FR_EMESH;
    }
    int code = F0.nc == 4 ? find_orientation(c0, F0.ref, c1, F1.ref, shift, tol)
                          : find_tri_orientation(c0, c1, shift, tol);
    if (code < 0) {
      err = "could not orient a matched face pair";
      return FR_EMESH;
    }
    orient[I] = code;
    if (Ep > 0) m.if_tri[I] = F0.nc == 3 ? 1 : 0;
    m.if_elem[2 * I] = (int32_t)pr.first.e;
    m.if_elem[2 * I + 1] = (int32_t)pr.second.e;
    set_ef(pr.first, (int32_t)((I << 4) | (0 << 3) | 0));
    set_ef(pr.second, (int32_t)((I << 4) | (1 << 3) | code));
  }
  for (size_t k = 0; k < bfaces.size(); ++k) {
    int64_t I = n_int + (int64_t)k;
    m.if_bc[I] = bfaces[k].second;
    m.if_elem[2 * I] = (int32_t)bfaces[k].first.e;
    if (Ep > 0) m.if_tri[I] = (bfaces[k].first.e >= E && bfaces[k].first.f < 2) ? 1 : 0;
    set_ef(bfaces[k].first, (int32_t)(I << 4));
  }
  for (int64_t i = 0; i < E * 6; ++i)
    if (m.ef[i] < 0) {
      err = "internal: element face without interface";
      return FR_EMESH;
    }
  for (int64_t i = 0; i < Ep * 5; ++i)
    if (m.ef_p[i] < 0) {
      err = "internal: element face without interface";
      return FR_EMESH;
    }

  // Geometry at solution and flux points, element by element on host threads (every element
  // writes only its own metrics, points and lift factors, and the normals of the interfaces whose
  // side 0 it is).
  Basis1D b = make_basis(p, vcjh_c);   // correction vectors enter the BR2 lift factors
  m.metrics.assign((size_t)E * 10 * Np, 0.0);
  m.liftfac.assign((size_t)E * 6 * 3 * Nf, 0.0);
  m.normals.assign((size_t)m.n_if * 4 * Nf, 0.0);
  m.xsol.assign(((size_t)E * Np + (size_t)Ep * Npp) * 3, 0.0);
  m.h.assign(G, 0.0);
  std::vector<double> fx((size_t)(E * 6 + Ep * 5) * Nf * 3);   // flux-point coordinates for the match check
  // Quadratic elements: positions and |J| from the element map, S from the curl form.
  const bool curved_h = hn == 27, curved_p = pn == 18;
  CurvedOps cops;
  if (curved_h || curved_p) curved_ops(p, b, Ep > 0 ? &tb : nullptr, cops);
  std::atomic<int64_t> bad_elem(INT64_MAX);
  auto store_normal = [&](int64_t I, int r, const double n[3]) {
    double nn = 0.0;
    for (int jj = 0; jj < 3; ++jj) {
      m.normals[((size_t)I * 4 + jj) * Nf + r] = n[jj];
      nn += n[jj] * n[jj];
    }
    m.normals[((size_t)I * 4 + 3) * Nf + r] = std::sqrt(nn);
  };
  auto note_bad = [&](int64_t g) {
    int64_t cur = bad_elem.load();
    while (g < cur && !bad_elem.compare_exchange_weak(cur, g)) {
    }
  };
  parallel_for(E, [&](int64_t e0, int64_t e1) {
    std::vector<double> xs((size_t)3 * Np), dets(Np), Ssol((size_t)9 * Np), xfc((size_t)6 * Nf * 3),
        Sface((size_t)6 * 9 * Nf);
    for (int64_t e = e0; e < e1; ++e) {
      double X[27][3];
      elem_verts(e, X, hn);
      if (curved_h) hex27_geometry(cops, X, xs.data(), dets.data(), Ssol.data(), xfc.data(), Sface.data());
      double vol = 0.0;
      double *met = &m.metrics[(size_t)e * 10 * Np];
      bool ok = true;
      for (int k = 0; k < N; ++k)
        for (int j = 0; j < N; ++j)
          for (int i = 0; i < N; ++i) {
            const int mm = i + N * j + N * N * k;
            double S[3][3], det, gx[3];
            if (curved_h) {
              det = dets[mm];
              for (int d = 0; d < 3; ++d)
                for (int jj = 0; jj < 3; ++jj) S[d][jj] = Ssol[(size_t)(d * 3 + jj) * Np + mm];
              for (int c = 0; c < 3; ++c) gx[c] = xs[(size_t)mm * 3 + c];
            } else {
              const double xi[3] = {b.x[i], b.x[j], b.x[k]};
              Jac g = trilinear(X, xi);
              adjugate_rows(g.J, S, det);
              for (int c = 0; c < 3; ++c) gx[c] = g.x[c];
            }
            if (!(det > 0.0)) ok = false;
            for (int d = 0; d < 3; ++d)
              for (int jj = 0; jj < 3; ++jj) met[(d * 3 + jj) * Np + mm] = S[d][jj];
            met[9 * Np + mm] = 1.0 / det;
            vol += b.w[i] * b.w[j] * b.w[k] * det;
            for (int c = 0; c < 3; ++c) m.xsol[((size_t)e * Np + mm) * 3 + c] = gx[c];
          }
      if (!ok) {
        note_bad(e);
        continue;
      }
      m.h[e] = std::cbrt(vol);
      for (int f = 0; f < 6; ++f) {
        int d, s, t0, t1;
        face_axes(f, d, s, t0, t1);
        const double *lv = (s > 0) ? b.lp : b.lm;
        const double *hv = (s > 0) ? b.hp : b.hm;
        const int packed = m.ef[e * 6 + f];
        const int64_t I = packed >> 4;
        const int side = (packed >> 3) & 1;
        for (int bb = 0; bb < N; ++bb)
          for (int aa = 0; aa < N; ++aa) {
            const int r = aa + N * bb;
            double acc[3] = {0, 0, 0};
            for (int c = 0; c < N; ++c) {
              int idx[3];
              idx[d] = c; idx[t0] = aa; idx[t1] = bb;
              const int mm = idx[0] + N * idx[1] + N * N * idx[2];
              for (int jj = 0; jj < 3; ++jj)
                acc[jj] += lv[c] * hv[c] * met[(d * 3 + jj) * Np + mm] * met[9 * Np + mm];
            }
            for (int jj = 0; jj < 3; ++jj)
              m.liftfac[(((size_t)e * 6 + f) * 3 + jj) * Nf + r] = s * acc[jj];
            double Sd[3], gx[3];
            if (curved_h) {
              for (int jj = 0; jj < 3; ++jj) Sd[jj] = Sface[((size_t)f * 9 + d * 3 + jj) * Nf + r];
              for (int c = 0; c < 3; ++c) gx[c] = xfc[((size_t)f * Nf + r) * 3 + c];
            } else {
              double xi[3], S[3][3], det;
              xi[d] = (double)s; xi[t0] = b.x[aa]; xi[t1] = b.x[bb];
              Jac g = trilinear(X, xi);
              adjugate_rows(g.J, S, det);
              for (int jj = 0; jj < 3; ++jj) Sd[jj] = S[d][jj];
              for (int c = 0; c < 3; ++c) gx[c] = g.x[c];
            }
            for (int c = 0; c < 3; ++c) fx[((size_t)face_index(e, f) * Nf + r) * 3 + c] = gx[c];
            if (side == 0) {
              const double n[3] = {s * Sd[0], s * Sd[1], s * Sd[2]};
              store_normal(I, r, n);
            }
          }
      }
    }
  });
  if (bad_elem.load() != INT64_MAX) {
    snprintf(buf, sizeof buf, "non-positive Jacobian in element %lld", (long long)bad_elem.load());
    err = buf;
    return FR_EMESH;
  }
  if (Ep > 0) {
    // Prisms: solution points (triangle node q, line point k) -> m = q + Nt k.
    m.metrics_p.assign((size_t)Ep * 10 * Npp, 0.0);
    parallel_for(Ep, [&](int64_t e0, int64_t e1) {
      std::vector<double> xs((size_t)3 * Npp), dets(Npp), Ssol((size_t)9 * Npp), xfc((size_t)5 * Nf * 3),
          Sface((size_t)5 * 9 * Nf);
      for (int64_t ep = e0; ep < e1; ++ep) {
        const int64_t g = E + ep;
        double X[18][3];
        prism_verts(ep, X, pn);
        if (curved_p) prism18_geometry(cops, tb, X, xs.data(), dets.data(), Ssol.data(), xfc.data(), Sface.data());
        double vol = 0.0;
        double *met = &m.metrics_p[(size_t)ep * 10 * Npp];
        bool ok = true;
        for (int k = 0; k < N; ++k)
          for (int q = 0; q < Nt; ++q) {
            const int mm = q + Nt * k;
            double S[3][3], det, gx[3];
            if (curved_p) {
              det = dets[mm];
              for (int d = 0; d < 3; ++d)
                for (int jj = 0; jj < 3; ++jj) S[d][jj] = Ssol[(size_t)(d * 3 + jj) * Npp + mm];
              for (int c = 0; c < 3; ++c) gx[c] = xs[(size_t)mm * 3 + c];
            } else {
              const double xi[3] = {tb.r[q], tb.s[q], b.x[k]};
              Jac jg = prism_map(X, xi);
              adjugate_rows(jg.J, S, det);
              for (int c = 0; c < 3; ++c) gx[c] = jg.x[c];
            }
            if (!(det > 0.0)) ok = false;
            for (int d = 0; d < 3; ++d)
              for (int jj = 0; jj < 3; ++jj) met[(d * 3 + jj) * Npp + mm] = S[d][jj];
            met[9 * Npp + mm] = 1.0 / det;
            vol += tb.wT[q] * b.w[k] * det;
            for (int c = 0; c < 3; ++c) m.xsol[((size_t)E * Np + (size_t)ep * Npp + mm) * 3 + c] = gx[c];
          }
        if (!ok) {
          note_bad(g);
          continue;
        }
        m.h[g] = std::cbrt(vol);
        for (int f = 0; f < 5; ++f) {
          const int packed = m.ef_p[ep * 5 + f];
          const int64_t I = packed >> 4;
          const int side = (packed >> 3) & 1;
          const int nq = f < 2 ? Nt : Nf;
          for (int r = 0; r < nq; ++r) {
            double S[3][3], gx[3];
            if (curved_p) {
              for (int d = 0; d < 3; ++d)
                for (int jj = 0; jj < 3; ++jj) S[d][jj] = Sface[((size_t)f * 9 + d * 3 + jj) * Nf + r];
              for (int c = 0; c < 3; ++c) gx[c] = xfc[((size_t)f * Nf + r) * 3 + c];
            } else {
              double xi[3], det;
              if (f < 2) {
                xi[0] = tb.r[r]; xi[1] = tb.s[r]; xi[2] = f == 0 ? -1.0 : 1.0;
              } else {
                tri_edge_point(f - 2, b.x[r % N], xi[0], xi[1]);
                xi[2] = b.x[r / N];
              }
              Jac jg = prism_map(X, xi);
              adjugate_rows(jg.J, S, det);
              for (int c = 0; c < 3; ++c) gx[c] = jg.x[c];
            }
            for (int c = 0; c < 3; ++c) fx[((size_t)face_index(g, f) * Nf + r) * 3 + c] = gx[c];
            if (side == 0) {
              double n[3];
              for (int jj = 0; jj < 3; ++jj) {
                n[jj] = 0.0;
                for (int d = 0; d < 3; ++d)
                  if (kPrismNormal[f][d] != 0.0) n[jj] += kPrismNormal[f][d] * S[d][jj];
              }
              store_normal(I, r, n);
            }
          }
        }
      }
    });
    if (bad_elem.load() != INT64_MAX) {
      snprintf(buf, sizeof buf, "non-positive Jacobian in element %lld", (long long)bad_elem.load());
      err = buf;
      return FR_EMESH;
    }
    // Operator table (prism_tab layout).
    const PrismTab L = prism_tab(N);
    m.ptab.assign(L.size, 0.0);
    double *t = m.ptab.data();
    for (int i = 0; i < Nt * Nt; ++i) {
      t[L.Dr + i] = tb.Dr[i];
      t[L.Ds + i] = tb.Ds[i];
    }
    // Own-flux correction of the quadrilateral faces (reference normals (0,-1,0), (1,1,0),
    // (-1,0,0) for edges 0, 1, 2): Drt = Dr - LQ1 E1 + LQ2 E2, Dst = Ds + LQ0 E0 - LQ1 E1.
    for (int i = 0; i < Nt; ++i)
      for (int j = 0; j < Nt; ++j) {
        long double c[3];
        for (int e = 0; e < 3; ++e) {
          long double acc = 0;
          for (int a = 0; a < N; ++a) acc += (long double)tb.LQ[e][(size_t)i * N + a] * tb.E[e][(size_t)a * Nt + j];
          c[e] = acc;
        }
        t[L.Drt + i * Nt + j] = (double)((long double)tb.Dr[(size_t)i * Nt + j] - c[1] + c[2]);
        t[L.Dst + i * Nt + j] = (double)((long double)tb.Ds[(size_t)i * Nt + j] + c[0] - c[1]);
      }
    for (int e = 0; e < 3; ++e) {
      for (int i = 0; i < N * Nt; ++i) t[L.E + e * N * Nt + i] = tb.E[e][i];
      for (int i = 0; i < Nt * N; ++i) t[L.LQ + e * Nt * N + i] = tb.LQ[e][i];
    }
    for (int i = 0; i < N; ++i) {
      for (int a = 0; a < N; ++a) {
        t[L.D1 + i * N + a] = b.D[i * N + a];
        t[L.D1t + i * N + a] = b.D[i * N + a] - b.hp[i] * b.lp[a] + b.hm[i] * b.lm[a];
      }
      t[L.lm + i] = b.lm[i];
      t[L.lp + i] = b.lp[i];
      t[L.hm + i] = b.hm[i];
      t[L.hp + i] = b.hp[i];
    }
    m.tri_slot = tb.perm;
  }
  // LDG switch per interface: side 0 supplies the common solution when its outward normal, summed
  // over the face's flux points, points along (1, sqrt(2)/2, sqrt(3)/4).
  m.if_up.assign(m.n_if, 0);
  {
    const double sw[3] = {1.0, std::sqrt(2.0) / 2.0, std::sqrt(3.0) / 4.0};
    for (int64_t I = 0; I < n_int; ++I) {
      const int nq = (Ep > 0 && m.if_tri[I]) ? Nt : Nf;
      double s = 0.0;
      for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
        for (int r = 0; r < nq; ++r) acc += m.normals[((size_t)I * 4 + c) * Nf + r];
        s += acc * sw[c];
      }
      m.if_up[I] = s > 0.0 ? 1 : 0;
    }
  }
  // Check that every side-1 flux point lands on its side-0 slot (coordinates, with shift).
  for (int64_t I = 0; I < n_int; ++I) {
    bool per = I >= (int64_t)pairs.size();
    const auto &pr = per ? ppairs[I - pairs.size()] : pairs[I];
    double shift[3] = {0, 0, 0};
    if (per)
      for (int i = 0; i < 3; ++i) shift[i] = pshift[I - pairs.size()][i];
    const bool tri = Ep > 0 && m.if_tri[I];
    const int nq = tri ? Nt : Nf;
    for (int r = 0; r < nq; ++r) {
      const int q = tri ? m.tri_slot[(size_t)orient[I] * Nt + r] : orient_slot(orient[I], r % N, r / N, N);
      const double *x1 = &fx[((size_t)face_index(pr.second.e, pr.second.f) * Nf + r) * 3];
      const double *x0 = &fx[((size_t)face_index(pr.first.e, pr.first.f) * Nf + q) * 3];
      double dd = 0;
      for (int c = 0; c < 3; ++c) dd += (x1[c] - shift[c] - x0[c]) * (x1[c] - shift[c] - x0[c]);
      if (dd > 1e4 * tol * tol) {
        err = "flux points of a matched face pair do not coincide";
        return FR_EMESH;
      }
    }
  }
  return FR_OK;
}

}  // namespace frx
