"""Triangle nodal basis for prism elements (oracle; test infrastructure only).

Reference triangle T = {(r, s): r >= -1, s >= -1, r + s <= 0}.  The paper's FR method (section "FR
Algorithm", Eq. 2) uses a nodal Lagrange basis on solution points; for the triangle layer of a
prism this build's reading takes:
  * nodes: the warp-and-blend construction of Warburton (2006) -- equidistant barycentric nodes
    warped along each edge by the displacement from equidistant to Gauss-Lobatto-Legendre points,
    blended into the interior, with the published optimised blend parameter alpha(p) -- a set that
    is symmetric under the triangle's six symmetries and unisolvent;
  * modal basis: the orthonormal Proriol-Koornwinder-Dubiner polynomials
    psi_ij(r, s) = sqrt(2) P~_i(a) (1 - s)^i P~_j^(2i+1,0)(s),  a = 2(1 + r)/(1 - s) - 1,
    P~ orthonormal Jacobi polynomials (scipy.special for the values);
  * derivatives from the chain rule through the collapse, written so that (1 - s)^(i-1) absorbs
    the 1/(1 - s) of da/dr and da/ds (at the top vertex s = 1, a = -1: the limit along r = -1).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import eval_jacobi, gammaln

# Optimised blend parameter alpha(p), p = 1..15 (Warburton 2006).
ALPHA_OPT = [0.0, 0.0, 1.4152, 0.1001, 0.2751, 0.9800, 1.0999, 1.2832, 1.3648, 1.4773, 1.4959, 1.5743, 1.5770,
             1.6223, 1.6258]


def jacobi_norm(x, n, a, b):
    """Orthonormal Jacobi polynomial on [-1, 1] with weight (1-x)^a (1+x)^b."""
    if n < 0:
        return np.zeros_like(np.asarray(x, dtype=np.float64))
    logh = (a + b + 1) * math.log(2.0) - math.log(2 * n + a + b + 1) + gammaln(n + a + 1) + gammaln(n + b + 1) \
        - gammaln(n + a + b + 1) - gammaln(n + 1)
    return eval_jacobi(n, a, b, x) / math.exp(0.5 * logh)


def jacobi_norm_deriv(x, n, a, b):
    """d/dx of the orthonormal Jacobi polynomial (via d/dx P_n^(a,b) = (n+a+b+1)/2 P_{n-1}^(a+1,b+1))."""
    if n == 0:
        return np.zeros_like(np.asarray(x, dtype=np.float64))
    logh = (a + b + 1) * math.log(2.0) - math.log(2 * n + a + b + 1) + gammaln(n + a + 1) + gammaln(n + b + 1) \
        - gammaln(n + a + b + 1) - gammaln(n + 1)
    return 0.5 * (n + a + b + 1) * eval_jacobi(n - 1, a + 1, b + 1, x) / math.exp(0.5 * logh)


def gauss_lobatto(N):
    """N+1 Gauss-Lobatto-Legendre points: -1, roots of P_N', 1."""
    if N == 1:
        return np.array([-1.0, 1.0])
    inner = np.sort(np.polynomial.legendre.Legendre.basis(N).deriv().roots().real)
    return np.concatenate([[-1.0], inner, [1.0]])


def nodes(p):
    """Warp-and-blend nodes of degree p on the reference triangle: [Nt][2] (r, s)."""
    Np = (p + 1) * (p + 2) // 2
    alpha = ALPHA_OPT[p - 1] if p <= 15 else 5.0 / 3.0
    L1, L3 = [], []
    for n in range(p + 1):
        for m in range(p + 1 - n):
            L1.append(n / p)
            L3.append(m / p)
    L1, L3 = np.array(L1), np.array(L3)
    L2 = 1.0 - L1 - L3
    x = -L2 + L3
    y = (-L2 - L3 + 2 * L1) / math.sqrt(3.0)
    req = np.linspace(-1.0, 1.0, p + 1)
    rlgl = gauss_lobatto(p)

    def warp(r):
        # displacement from equidistant to LGL points, interpolated at r, divided by (1 - r^2)
        w = np.zeros_like(r)
        for i in range(p + 1):
            li = np.ones_like(r)
            for j in range(p + 1):
                if j != i:
                    li *= (r - req[j]) / (req[i] - req[j])
            w += li * (rlgl[i] - req[i])
        zerof = np.abs(r) < 1.0 - 1e-10
        return np.where(zerof, w / np.where(zerof, 1.0 - r * r, 1.0), 0.0)

    b1, b2, b3 = 4 * L2 * L3, 4 * L1 * L3, 4 * L1 * L2
    w1, w2, w3 = warp(L3 - L2), warp(L1 - L3), warp(L2 - L1)
    f1 = b1 * w1 * (1 + (alpha * L1) ** 2)
    f2 = b2 * w2 * (1 + (alpha * L2) ** 2)
    f3 = b3 * w3 * (1 + (alpha * L3) ** 2)
    X = x + f1 + math.cos(2 * math.pi / 3) * f2 + math.cos(4 * math.pi / 3) * f3
    Y = y + math.sin(2 * math.pi / 3) * f2 + math.sin(4 * math.pi / 3) * f3
    # equilateral (X, Y) -> reference (r, s) via barycentric coordinates
    l1 = (math.sqrt(3.0) * Y + 1.0) / 3.0
    l2 = (-3.0 * X - math.sqrt(3.0) * Y + 2.0) / 6.0
    l3 = (3.0 * X - math.sqrt(3.0) * Y + 2.0) / 6.0
    r = -l2 + l3 - l1
    s = -l2 - l3 + l1
    out = np.stack([r, s], axis=1)
    assert out.shape[0] == Np
    return out


def _collapse(rs):
    r, s = rs[:, 0], rs[:, 1]
    top = np.abs(1.0 - s) < 1e-12
    a = np.where(top, -1.0, 2.0 * (1.0 + r) / np.where(top, 1.0, 1.0 - s) - 1.0)
    return a, s


def modes(p):
    return [(i, j) for i in range(p + 1) for j in range(p + 1 - i)]


def vandermonde(p, rs):
    """V[q][n] = psi_n(r_q, s_q) (orthonormal on T)."""
    a, s = _collapse(rs)
    cols = [math.sqrt(2.0) * jacobi_norm(a, i, 0, 0) * (1.0 - s) ** i * jacobi_norm(s, j, 2 * i + 1, 0)
            for (i, j) in modes(p)]
    return np.stack(cols, axis=1)


def grad_vandermonde(p, rs):
    """(Vr, Vs) with the r and s derivatives of every mode at the points."""
    a, s = _collapse(rs)
    Vr, Vs = [], []
    for (i, j) in modes(p):
        fa, dfa = jacobi_norm(a, i, 0, 0), jacobi_norm_deriv(a, i, 0, 0)
        gb, dgb = jacobi_norm(s, j, 2 * i + 1, 0), jacobi_norm_deriv(s, j, 2 * i + 1, 0)
        u_im1 = (1.0 - s) ** (i - 1) if i >= 1 else np.zeros_like(s)
        dr = 2.0 * dfa * u_im1 * gb
        ds = dfa * (1.0 + a) * u_im1 * gb + fa * (-i * u_im1 * gb + (1.0 - s) ** i * dgb)
        Vr.append(math.sqrt(2.0) * dr)
        Vs.append(math.sqrt(2.0) * ds)
    return np.stack(Vr, axis=1), np.stack(Vs, axis=1)


class Tri:
    """Nodal operators of the degree-p triangle on the warp-and-blend nodes."""

    def __init__(self, p):
        self.p = p
        self.rs = nodes(p)
        self.Nt = self.rs.shape[0]
        self.V = vandermonde(p, self.rs)
        self.Vinv = np.linalg.inv(self.V)
        Vr, Vs = grad_vandermonde(p, self.rs)
        self.Dr = Vr @ self.Vinv
        self.Ds = Vs @ self.Vinv
        self.M = self.Vinv.T @ self.Vinv          # exact mass matrix (orthonormal modes)

    def interp(self, pts):
        """Lagrange basis values at pts: [len(pts)][Nt]."""
        return vandermonde(self.p, np.asarray(pts, dtype=np.float64)) @ self.Vinv
