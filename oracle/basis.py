"""1D building blocks of the FR discretisation (oracle; test infrastructure only).

Eq. 2a-c of arXiv 2308.06605 represent Q, F and G by Lagrange polynomials l_i through the
solution points; the hexahedral element uses their tensor products.  This module gives, for the
Gauss-Legendre point set:
  * the nodes and weights (Newton iteration on the Legendre polynomial P_N from Chebyshev-like
    starting guesses),
  * Lagrange values l_j(x) as the literal product formula,
  * derivative values l_j'(x) by the product rule applied term by term,
  * the DG-equivalent correction function of the section "FR Algorithm": g is the right Radau
    polynomial g_R = (P_N + P_{N-1})/2 (g_R(1) = 1, g_R(-1) = 0, orthogonal to degree N-2),
    g_L(x) = g_R(-x).  Its derivative comes from the Legendre derivative recurrence.
"""
from __future__ import annotations

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


def correction_right(N: int, x):
    """g_R(x) = (P_N(x) + P_{N-1}(x)) / 2, the right Radau polynomial (DG-equivalent, c = 0)."""
    PN, _ = legendre(N, x)
    PM, _ = legendre(N - 1, x)
    return 0.5 * (PN + PM)


def correction_right_derivative(N: int, x):
    """g_R'(x) = (P_N'(x) + P_{N-1}'(x)) / 2."""
    _, dPN = legendre(N, x)
    _, dPM = legendre(N - 1, x)
    return 0.5 * (dPN + dPM)


class Basis1D:
    """All 1D arrays of an order-p GL element (N = p + 1 points)."""

    def __init__(self, p: int):
        self.p = p
        self.N = N = p + 1
        self.nodes, self.weights = gauss_legendre(N)
        self.D = derivative_matrix(self.nodes)                          # [N][N]
        self.l_minus = lagrange_values(self.nodes, [-1.0])[0]           # l_j(-1)
        self.l_plus = lagrange_values(self.nodes, [1.0])[0]             # l_j(+1)
        # Derivative of the correction attached to a face, evaluated at the solution points,
        # as a function of the outward sign s of that face: h_s(xi_i) = g_R'(s * xi_i).
        self.h_plus = correction_right_derivative(N, self.nodes)
        self.h_minus = correction_right_derivative(N, -self.nodes)
