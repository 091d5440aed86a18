// Nodal triangle basis of the prism elements, computed in long double on the host.
//
// The FR method (section "FR Algorithm", Eq. 2) represents the solution by a nodal Lagrange basis
// on the solution points.  On the triangle layer of a prism the points are the warp-and-blend
// nodes of Warburton (2006): equidistant barycentric nodes moved along each edge by the
// displacement between equidistant and Gauss-Lobatto-Legendre points on that edge, blended into
// the interior with the published optimised blend parameter alpha(p).  Operators come from the
// orthonormal Proriol-Koornwinder-Dubiner modes
//   psi_ij(r, s) = sqrt(2) P~_i(a) P~_j^(2i+1,0)(s) (1 - s)^i,   a = 2 (1 + r) / (1 - s) - 1,
// through the Vandermonde matrix V[q][n] = psi_n(node q): D_r = V_r V^-1, D_s = V_s V^-1,
// M^-1 = V V^T, interpolation to edge points psi(x) V^-1.
#include <algorithm>
#include <cmath>

#include "fr_internal.hpp"

namespace frx {

using ld = long double;

namespace {

// Optimised blend parameter alpha(p), p = 1..15 (Warburton 2006, table of alpha_opt).
constexpr double kAlphaOpt[15] = {0.0000, 0.0000, 1.4152, 0.1001, 0.2751, 0.9800, 1.0999, 1.2832,
                                  1.3648, 1.4773, 1.4959, 1.5743, 1.5770, 1.6223, 1.6258};

// Orthonormal Jacobi polynomials P~_0..P~_n^(al,be) at x by the three-term recurrence of the
// orthonormal family (weight (1-x)^al (1+x)^be on [-1, 1]).
ld jacobi_orth(ld x, int n, int al, int be) {
  const ld a = al, b = be;
  const ld p0 = sqrtl(powl(2.0L, -a - b - 1.0L) * tgammal(a + b + 2.0L) / (tgammal(a + 1.0L) * tgammal(b + 1.0L)));
  if (n == 0) return p0;
  ld pm = p0;
  ld pc = p0 * ((a + b + 2.0L) * x / 2.0L + (a - b) / 2.0L) * sqrtl((a + b + 3.0L) / ((a + 1.0L) * (b + 1.0L)));
  ld aold = 2.0L / (2.0L + a + b) * sqrtl((a + 1.0L) * (b + 1.0L) / (a + b + 3.0L));
  for (int i = 1; i < n; ++i) {
    const ld h1 = 2.0L * i + a + b;
    const ld anew = 2.0L / (h1 + 2.0L) *
                    sqrtl((i + 1.0L) * (i + 1.0L + a + b) * (i + 1.0L + a) * (i + 1.0L + b) / ((h1 + 1.0L) * (h1 + 3.0L)));
    const ld bnew = -(a * a - b * b) / (h1 * (h1 + 2.0L));
    const ld pn = (-aold * pm + (x - bnew) * pc) / anew;
    pm = pc;
    pc = pn;
    aold = anew;
  }
  return pc;
}

// d/dx P~_n^(al,be) = sqrt(n (n + al + be + 1)) P~_{n-1}^(al+1,be+1).
ld jacobi_orth_d(ld x, int n, int al, int be) {
  if (n == 0) return 0.0L;
  return sqrtl((ld)n * (n + al + be + 1)) * jacobi_orth(x, n - 1, al + 1, be + 1);
}

ld ipow(ld x, int k) {
  ld r = 1.0L;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

// Gauss-Lobatto-Legendre points of degree p: -1, the roots of P_p', +1 (Newton from the
// Chebyshev-Gauss-Lobatto points, with P_p'' from the Legendre equation).
void gll_points(int p, ld *x) {
  x[0] = -1.0L;
  x[p] = 1.0L;
  for (int j = 1; j < p; ++j) {
    ld t = -cosl(3.14159265358979323846264338327950288L * j / p);
    for (int it = 0; it < 100; ++it) {
      ld P0 = 1.0L, P1 = t;
      for (int k = 1; k < p; ++k) {
        const ld P2 = ((2 * k + 1) * t * P1 - k * P0) / (k + 1);
        P0 = P1;
        P1 = P2;
      }
      const ld dP = p * (P0 - t * P1) / (1.0L - t * t);
      const ld d2P = (2.0L * t * dP - p * (p + 1.0L) * P1) / (1.0L - t * t);
      const ld step = dP / d2P;
      t -= step;
      if (fabsl(step) < 1e-30L) break;
    }
    x[j] = t;
  }
  std::sort(x, x + p + 1);
}

struct Modes {
  int n;
  int i[64], j[64];
};

Modes modes_of(int p) {
  Modes m{};
  for (int i = 0; i <= p; ++i)
    for (int j = 0; j <= p - i; ++j) {
      m.i[m.n] = i;
      m.j[m.n] = j;
      ++m.n;
    }
  return m;
}

// psi_n and its r, s derivatives at (r, s).
void eval_modes(const Modes &M, ld r, ld s, ld *v, ld *vr, ld *vs) {
  const bool top = fabsl(1.0L - s) < 1e-14L;
  const ld a = top ? -1.0L : 2.0L * (1.0L + r) / (1.0L - s) - 1.0L;
  const ld sq2 = sqrtl(2.0L);
  for (int n = 0; n < M.n; ++n) {
    const int i = M.i[n], j = M.j[n];
    const ld fa = jacobi_orth(a, i, 0, 0), dfa = jacobi_orth_d(a, i, 0, 0);
    const ld gb = jacobi_orth(s, j, 2 * i + 1, 0), dgb = jacobi_orth_d(s, j, 2 * i + 1, 0);
    const ld u_i = ipow(1.0L - s, i);
    const ld u_im1 = i >= 1 ? ipow(1.0L - s, i - 1) : 0.0L;
    if (v) v[n] = sq2 * fa * gb * u_i;
    if (vr) vr[n] = sq2 * 2.0L * dfa * gb * u_im1;
    if (vs) vs[n] = sq2 * (dfa * (1.0L + a) * gb * u_im1 + fa * (dgb * u_i - i * gb * u_im1));
  }
}

// In-place inverse of the n x n matrix A (Gauss-Jordan with partial pivoting).
bool invert(std::vector<ld> &A, int n) {
  std::vector<ld> B((size_t)n * n, 0.0L);
  for (int i = 0; i < n; ++i) B[(size_t)i * n + i] = 1.0L;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(A[(size_t)r * n + c]) > fabsl(A[(size_t)piv * n + c])) piv = r;
    if (fabsl(A[(size_t)piv * n + c]) < 1e-300L) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
        std::swap(B[(size_t)c * n + k], B[(size_t)piv * n + k]);
      }
    const ld d = A[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) {
      A[(size_t)c * n + k] /= d;
      B[(size_t)c * n + k] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const ld f = A[(size_t)r * n + c];
      if (f == 0.0L) continue;
      for (int k = 0; k < n; ++k) {
        A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
        B[(size_t)r * n + k] -= f * B[(size_t)c * n + k];
      }
    }
  }
  A.swap(B);
  return true;
}

}  // namespace

// Vertex permutations of a triangular face: code c maps corner a of one side to corner
// kTriPerm[c][a] of the other.
const int kTriPerm[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};

void tri_edge_point(int edge, double sigma, double &r, double &s) {
  switch (edge) {
    case 0: r = sigma; s = -1.0; break;     // s = -1, from vertex 0 to vertex 1
    case 1: r = -sigma; s = sigma; break;   // r + s = 0, from vertex 1 to vertex 2
    default: r = -1.0; s = -sigma; break;   // r = -1, from vertex 2 to vertex 0
  }
}

bool tri_transfer(int p, int q, std::vector<double> &T) {
  TriBasis bp, bq;
  if (!make_tri_basis(p, bp) || !make_tri_basis(q, bq)) return false;
  const Modes Mp = modes_of(p), Mq = modes_of(q);
  const int np = Mp.n, nq = Mq.n;
  std::vector<ld> Vp((size_t)np * np), row(np), rowq(nq);
  for (int k = 0; k < np; ++k) eval_modes(Mp, (ld)bp.r[k], (ld)bp.s[k], &Vp[(size_t)k * np], nullptr, nullptr);
  if (!invert(Vp, np)) return false;          // modal coefficients from nodal values
  T.assign((size_t)nq * np, 0.0);
  for (int t = 0; t < nq; ++t) {
    eval_modes(Mq, (ld)bq.r[t], (ld)bq.s[t], rowq.data(), nullptr, nullptr);
    for (int j = 0; j < np; ++j) {
      ld acc = 0;
      for (int n = 0; n < np; ++n) {
        if (Mp.i[n] + Mp.j[n] > q) continue;  // modes above the target degree are dropped
        int nn = -1;
        for (int k = 0; k < nq; ++k)
          if (Mq.i[k] == Mp.i[n] && Mq.j[k] == Mp.j[n]) nn = k;
        acc += rowq[nn] * Vp[(size_t)n * np + j];
      }
      T[(size_t)t * np + j] = (double)acc;
    }
  }
  return true;
}

void gll_nodes(int p, double *x) {
  ld t[kMaxN + 1];
  gll_points(p, t);
  for (int i = 0; i <= p; ++i) x[i] = (double)t[i];
}

bool make_tri_basis(int p, TriBasis &T) {
  const int N = p + 1, Nt = N * (N + 1) / 2;
  T.p = p;
  T.N = N;
  T.Nt = Nt;
  // --- warp-and-blend nodes
  const ld alpha = p <= 15 ? (ld)kAlphaOpt[p - 1] : 5.0L / 3.0L;
  ld req[kMaxN], rgll[kMaxN];
  for (int i = 0; i <= p; ++i) req[i] = -1.0L + 2.0L * i / p;
  gll_points(p, rgll);
  auto warp = [&](ld r) {
    ld w = 0.0L;
    for (int i = 0; i <= p; ++i) {
      ld li = 1.0L;
      for (int j = 0; j <= p; ++j)
        if (j != i) li *= (r - req[j]) / (req[i] - req[j]);
      w += li * (rgll[i] - req[i]);
    }
    return fabsl(r) < 1.0L - 1e-10L ? w / (1.0L - r * r) : 0.0L;
  };
  const ld s3 = sqrtl(3.0L), pi = 3.14159265358979323846264338327950288L;
  T.r.assign(Nt, 0.0);
  T.s.assign(Nt, 0.0);
  std::vector<ld> rl(Nt), sl(Nt);
  int q = 0;
  for (int n = 0; n <= p; ++n)
    for (int m = 0; m <= p - n; ++m, ++q) {
      const ld L1 = (ld)n / p, L3 = (ld)m / p, L2 = 1.0L - L1 - L3;
      const ld x = -L2 + L3, y = (-L2 - L3 + 2.0L * L1) / s3;
      const ld f1 = 4.0L * L2 * L3 * warp(L3 - L2) * (1.0L + (alpha * L1) * (alpha * L1));
      const ld f2 = 4.0L * L1 * L3 * warp(L1 - L3) * (1.0L + (alpha * L2) * (alpha * L2));
      const ld f3 = 4.0L * L1 * L2 * warp(L2 - L1) * (1.0L + (alpha * L3) * (alpha * L3));
      const ld X = x + f1 + cosl(2.0L * pi / 3.0L) * f2 + cosl(4.0L * pi / 3.0L) * f3;
      const ld Y = y + sinl(2.0L * pi / 3.0L) * f2 + sinl(4.0L * pi / 3.0L) * f3;
      const ld l1 = (s3 * Y + 1.0L) / 3.0L, l2 = (-3.0L * X - s3 * Y + 2.0L) / 6.0L,
               l3 = (3.0L * X - s3 * Y + 2.0L) / 6.0L;
      rl[q] = -l2 + l3 - l1;
      sl[q] = -l2 - l3 + l1;
      T.r[q] = (double)rl[q];
      T.s[q] = (double)sl[q];
    }
  // --- Vandermonde, inverse, derivative matrices, inverse mass matrix
  const Modes M = modes_of(p);
  if (M.n != Nt) return false;
  std::vector<ld> V((size_t)Nt * Nt), Vr((size_t)Nt * Nt), Vs((size_t)Nt * Nt);
  for (int k = 0; k < Nt; ++k) eval_modes(M, rl[k], sl[k], &V[(size_t)k * Nt], &Vr[(size_t)k * Nt], &Vs[(size_t)k * Nt]);
  std::vector<ld> Vi = V;
  if (!invert(Vi, Nt)) return false;
  T.Dr.assign((size_t)Nt * Nt, 0.0);
  T.Ds.assign((size_t)Nt * Nt, 0.0);
  T.Minv.assign((size_t)Nt * Nt, 0.0);
  std::vector<ld> Mass((size_t)Nt * Nt, 0.0L);
  for (int i = 0; i < Nt; ++i)
    for (int j = 0; j < Nt; ++j) {
      ld dr = 0, ds = 0, mi = 0, ms = 0;
      for (int n = 0; n < Nt; ++n) {
        dr += Vr[(size_t)i * Nt + n] * Vi[(size_t)n * Nt + j];
        ds += Vs[(size_t)i * Nt + n] * Vi[(size_t)n * Nt + j];
        mi += V[(size_t)i * Nt + n] * V[(size_t)j * Nt + n];
        ms += Vi[(size_t)n * Nt + i] * Vi[(size_t)n * Nt + j];
      }
      T.Dr[(size_t)i * Nt + j] = (double)dr;
      T.Ds[(size_t)i * Nt + j] = (double)ds;
      T.Minv[(size_t)i * Nt + j] = (double)mi;
      Mass[(size_t)i * Nt + j] = ms;
    }
  T.wT.assign(Nt, 0.0);
  for (int i = 0; i < Nt; ++i) {
    ld acc = 0;
    for (int j = 0; j < Nt; ++j) acc += Mass[(size_t)i * Nt + j];
    T.wT[i] = (double)acc;
  }
  // --- edge interpolation (Gauss-Legendre points of the line) and DG lifting M^-1 E^T diag(w)
  const Basis1D b = make_basis(p);
  std::vector<ld> ps(Nt);
  for (int e = 0; e < 3; ++e) {
    T.E[e].assign((size_t)N * Nt, 0.0);
    T.LQ[e].assign((size_t)Nt * N, 0.0);
    std::vector<ld> El((size_t)N * Nt, 0.0L);
    for (int a = 0; a < N; ++a) {
      double r, s;
      tri_edge_point(e, b.x[a], r, s);
      eval_modes(M, (ld)r, (ld)s, ps.data(), nullptr, nullptr);
      for (int j = 0; j < Nt; ++j) {
        ld acc = 0;
        for (int n = 0; n < Nt; ++n) acc += ps[n] * Vi[(size_t)n * Nt + j];
        El[(size_t)a * Nt + j] = acc;
        T.E[e][(size_t)a * Nt + j] = (double)acc;
      }
    }
    for (int i = 0; i < Nt; ++i)
      for (int a = 0; a < N; ++a) {
        ld acc = 0;
        for (int j = 0; j < Nt; ++j) {
          ld mij = 0;
          for (int n = 0; n < Nt; ++n) mij += V[(size_t)i * Nt + n] * V[(size_t)j * Nt + n];
          acc += mij * El[(size_t)a * Nt + j];
        }
        T.LQ[e][(size_t)i * N + a] = (double)(acc * (ld)b.w[a]);
      }
  }
  // --- node permutations under the six vertex permutations (the node set is symmetric)
  T.perm.assign((size_t)6 * Nt, -1);
  for (int c = 0; c < 6; ++c)
    for (int k = 0; k < Nt; ++k) {
      const ld lam[3] = {-(rl[k] + sl[k]) / 2.0L, (1.0L + rl[k]) / 2.0L, (1.0L + sl[k]) / 2.0L};
      ld lam2[3];
      for (int a = 0; a < 3; ++a) lam2[kTriPerm[c][a]] = lam[a];
      const ld r2 = 2.0L * lam2[1] - 1.0L, s2 = 2.0L * lam2[2] - 1.0L;
      int best = -1;
      ld bd = 1e300L;
      for (int k2 = 0; k2 < Nt; ++k2) {
        const ld d = fabsl(rl[k2] - r2) + fabsl(sl[k2] - s2);
        if (d < bd) { bd = d; best = k2; }
      }
      if (bd > 1e-12L) return false;
      T.perm[(size_t)c * Nt + k] = best;
    }
  return true;
}

}  // namespace frx

extern "C" fr_status fr_tri_basis(int32_t p, double *rs, double *Dr, double *Ds, double *Minv) {
  if (p < 1 || p > 7) return FR_EINVAL;
  frx::TriBasis T;
  if (!frx::make_tri_basis(p, T)) return FR_EINVAL;
  const size_t Nt = (size_t)T.Nt;
  for (size_t i = 0; i < Nt; ++i) {
    if (rs) {
      rs[2 * i] = T.r[i];
      rs[2 * i + 1] = T.s[i];
    }
    for (size_t j = 0; j < Nt; ++j) {
      if (Dr) Dr[i * Nt + j] = T.Dr[i * Nt + j];
      if (Ds) Ds[i * Nt + j] = T.Ds[i * Nt + j];
      if (Minv) Minv[i * Nt + j] = T.Minv[i * Nt + j];
    }
  }
  return FR_OK;
}
