"""1D building blocks of the FR discretisation (oracle; test infrastructure only).

Eq. 2a-c of arXiv 2308.06605 represent Q, F and G by Lagrange polynomials l_i through the
solution points; the hexahedral element uses their tensor products.  This module gives, for the
Gauss-Legendre point set:
  * the nodes and weights (Newton iteration on the Legendre polynomial P_N from Chebyshev-like
    starting guesses),
  * Lagrange values l_j(x) as the literal product formula,
  * derivative values l_j'(x) by the product rule applied term by term,
  * the correction function of the section "FR Algorithm".  The paper takes the DG-equivalent
    one, the right Radau polynomial g_R = (P_N + P_{N-1})/2 (g_R(1) = 1, g_R(-1) = 0, orthogonal
    to degree N-2), g_L(x) = g_R(-x).  The energy-stable family of Vincent, Castonguay & Jameson
    (J. Sci. Comput. 47, 2011) generalises it with one parameter c (c = 0: the Radau choice):
    for degree p = N - 1,
        g_L = (-1)^p / 2 [P_p - (eta P_{p-1} + P_{p+1}) / (1 + eta)],
        eta = c (2p + 1) (a_p p!)^2 / 2,   a_p = (2p)! / (2^p (p!)^2),
    which by P_k(-x) = (-1)^k P_k(x) is, mirrored,
        g_R(x) = g_L(-x) = [P_p + (eta P_{p-1} + P_{p+1}) / (1 + eta)] / 2.
    The family needs 1 + eta > 0.  Derivatives come from the Legendre derivative recurrence.
"""
from __future__ import annotations

import math

import numpy as np


def legendre(n: int, x):
    """P_n(x) and P_n'(x) by the three-term recurrences
    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} and P'_{k+1} = P'_{k-1} + (2k+1) P_k."""
    x = np.asarray(x, dtype=np.float64)
    P = [np.ones_like(x), x.copy()]
    dP = [np.zeros_like(x), np.ones_like(x)]
    for k in range(1, n):
        P.append(((2 * k + 1) * x * P[k] - k * P[k - 1]) / (k + 1))
        dP.append(dP[k - 1] + (2 * k + 1) * P[k])
    return P[n], dP[n]


def gauss_legendre(N: int):
    """N Gauss-Legendre nodes (ascending) and weights on [-1, 1]."""
    i = np.arange(1, N + 1)
    x = np.cos(np.pi * (i - 0.25) / (N + 0.5))
    for _ in range(100):
        P, dP = legendre(N, x)
        dx = P / dP
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    P, dP = legendre(N, x)
    w = 2.0 / ((1.0 - x * x) * dP * dP)
    order = np.argsort(x)
    return x[order], w[order]


def lagrange_values(nodes, x):
    """L[q, j] = l_j(x_q) = prod_{m != j} (x_q - xi_m) / (xi_j - xi_m)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    N = len(nodes)
    L = np.ones((len(x), N))
    for j in range(N):
        for m in range(N):
            if m != j:
                L[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return L


def lagrange_derivatives(nodes, x):
    """Dl[q, j] = l_j'(x_q) = sum_{k != j} 1/(xi_j - xi_k) prod_{m != j,k} (x_q - xi_m)/(xi_j - xi_m)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    N = len(nodes)
    Dl = np.zeros((len(x), N))
    for j in range(N):
        for k in range(N):
            if k == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[k]))
            for m in range(N):
                if m != j and m != k:
                    term *= (x - nodes[m]) / (nodes[j] - nodes[m])
            Dl[:, j] += term
    return Dl


def derivative_matrix(nodes):
    """D[i, j] = l_j'(xi_i): derivative at the solution points of the nodal interpolant."""
    return lagrange_derivatives(nodes, nodes)


def vcjh_eta(p: int, c: float) -> float:
    """eta_p = c (2p + 1) (a_p p!)^2 / 2 with a_p = (2p)! / (2^p (p!)^2), the leading coefficient
    of P_p; raises if 1 + eta <= 0 (outside the family)."""
    a_p = math.factorial(2 * p) / (2.0 ** p * math.factorial(p) ** 2)
    eta = c * (2 * p + 1) * (a_p * math.factorial(p)) ** 2 / 2.0
    if not np.isfinite(eta) or 1.0 + eta <= 0.0:
        raise ValueError(f"VCJH parameter c = {c} is outside the family at p = {p} (1 + eta <= 0)")
    return eta


def correction_right(N: int, x, c: float = 0.0):
    """g_R(x) = [P_p + (eta P_{p-1} + P_{p+1}) / (1 + eta)] / 2, p = N - 1; c = 0 gives the
    right Radau polynomial (P_N + P_{N-1}) / 2 (DG-equivalent)."""
    p = N - 1
    eta = vcjh_eta(p, c)
    Pp, _ = legendre(p, x)
    Pm, _ = legendre(p - 1, x) if p >= 1 else (np.zeros_like(np.asarray(x, dtype=np.float64)), None)
    Pq, _ = legendre(p + 1, x)
    return 0.5 * (Pp + (eta * Pm + Pq) / (1.0 + eta))


def correction_right_derivative(N: int, x, c: float = 0.0):
    """g_R'(x) of `correction_right`, term by term."""
    p = N - 1
    eta = vcjh_eta(p, c)
    _, dPp = legendre(p, x)
    _, dPm = legendre(p - 1, x) if p >= 1 else (None, np.zeros_like(np.asarray(x, dtype=np.float64)))
    _, dPq = legendre(p + 1, x)
    return 0.5 * (dPp + (eta * dPm + dPq) / (1.0 + eta))


class Basis1D:
    """All 1D arrays of an order-p GL element (N = p + 1 points)."""

    def __init__(self, p: int, c: float = 0.0):
        self.p = p
        self.c = c
        self.N = N = p + 1
        self.nodes, self.weights = gauss_legendre(N)
        self.D = derivative_matrix(self.nodes)                          # [N][N]
        self.l_minus = lagrange_values(self.nodes, [-1.0])[0]           # l_j(-1)
        self.l_plus = lagrange_values(self.nodes, [1.0])[0]             # l_j(+1)
        # Derivative of the correction attached to a face, evaluated at the solution points,
        # as a function of the outward sign s of that face: h_s(xi_i) = g_R'(s * xi_i).
        self.h_plus = correction_right_derivative(N, self.nodes, c)
        self.h_minus = correction_right_derivative(N, -self.nodes, c)
