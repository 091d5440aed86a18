"""Pins of the oracle's 1D building blocks against what the mathematics fixes (CPU only)."""
import math
import os

import numpy as np
import pytest

from oracle import basis
from oracle.fr1d import residual_advection

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gauss_legendre_closed_forms.txt")


def _closed_forms():
    rows = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            n, x, w = (s.strip() for s in line.split(";"))
            env = {"sqrt": math.sqrt}
            rows.setdefault(int(n), []).append((eval(x, env), eval(w, env)))
    return rows


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_gauss_legendre_closed_forms(N):
    x, w = basis.gauss_legendre(N)
    want = []
    for xv, wv in _closed_forms()[N]:
        want.append((xv, wv))
        if xv != 0:
            want.append((-xv, wv))
    want.sort()
    np.testing.assert_allclose(x, [a for a, _ in want], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [b for _, b in want], rtol=2e-15, atol=0)


@pytest.mark.parametrize("N", range(1, 10))
def test_gauss_legendre_library_and_exactness(N):
    x, w = basis.gauss_legendre(N)
    xr, wr = np.polynomial.legendre.leggauss(N)
    np.testing.assert_allclose(x, xr, atol=1e-15)
    np.testing.assert_allclose(w, wr, rtol=1e-14)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * N):          # degree 2N-1 integrated exactly
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14


@pytest.mark.parametrize("p", range(1, 8))
def test_lagrange_and_derivative_exactness(p):
    N = p + 1
    x, _ = basis.gauss_legendre(N)
    L = basis.lagrange_values(x, x)
    np.testing.assert_allclose(L, np.eye(N), atol=1e-14)
    D = basis.derivative_matrix(x)
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-12)
    pts = np.linspace(-1, 1, 7)
    Lp = basis.lagrange_values(x, pts)
    Dp = basis.lagrange_derivatives(x, pts)
    for k in range(p + 1):           # degree <= p reproduced exactly, with derivatives
        np.testing.assert_allclose(D @ x ** k, k * x ** max(k - 1, 0) if k else 0 * x, atol=1e-11)
        np.testing.assert_allclose(Lp @ x ** k, pts ** k, atol=1e-13)
        np.testing.assert_allclose(Dp @ x ** k, k * pts ** max(k - 1, 0) if k else 0 * pts, atol=1e-11)


@pytest.mark.parametrize("p", range(1, 8))
def test_correction_function_identities(p):
    """g_R = right Radau: g_R(1)=1, g_R(-1)=0, orthogonal to P_{<=p-1}; and on GL points its
    derivative equals the DG lifting l_i(1)/w_i (the c = 0 equivalence)."""
    N = p + 1
    x, w = basis.gauss_legendre(N)
    assert abs(basis.correction_right(N, np.array([1.0]))[0] - 1.0) < 1e-14
    assert abs(basis.correction_right(N, np.array([-1.0]))[0]) < 1e-14
    xq, wq = np.polynomial.legendre.leggauss(N + 4)
    g = basis.correction_right(N, xq)
    for k in range(p):
        assert abs(np.sum(wq * g * xq ** k)) < 1e-14
    lp = basis.lagrange_values(x, [1.0])[0]
    np.testing.assert_allclose(basis.correction_right_derivative(N, x), lp / w, rtol=1e-12, atol=1e-12)
    assert abs(np.sum(w * basis.correction_right_derivative(N, x)) - 1.0) < 1e-13
    # derivative vs a centred finite difference of g_R itself
    hfd = 1e-6
    fd = (basis.correction_right(N, x + hfd) - basis.correction_right(N, x - hfd)) / (2 * hfd)
    np.testing.assert_allclose(basis.correction_right_derivative(N, x), fd, rtol=1e-7, atol=1e-7)
    b = basis.Basis1D(p)
    np.testing.assert_allclose(b.h_minus, b.h_plus[::-1], atol=1e-13)


def _modal_dg_residual(u_nodal, a, h, p):
    """Independent modal Legendre DG for u_t + a u_x = 0 on a periodic mesh (upwind flux).

    (h/2) 2/(2k+1) du_k/dt = a sum_l u_l int P_k' P_l - (P_k(1) f_R - P_k(-1) f_L), with
    int_{-1}^{1} P_k' P_l = 2 if k > l and k + l odd, else 0 (closed form)."""
    N = p + 1
    x, _ = basis.gauss_legendre(N)
    V = np.polynomial.legendre.legvander(x, p)          # V[i,k] = P_k(x_i)
    uh = np.linalg.solve(V, u_nodal.T).T                # [K][N] modal
    S = np.array([[2.0 if (k > l and (k + l) % 2 == 1) else 0.0 for l in range(N)] for k in range(N)])
    Pp = np.ones(N)
    Pm = np.array([(-1.0) ** k for k in range(N)])
    right = uh @ Pp
    left = uh @ Pm
    if a >= 0:
        fR = a * right
        fL = a * np.roll(right, 1)
    else:
        fR = a * np.roll(left, -1)
        fL = a * left
    rhs = a * uh @ S.T - np.outer(fR, Pp) + np.outer(fL, Pm)
    mass = (h / 2.0) * 2.0 / (2 * np.arange(N) + 1)
    duh = rhs / mass
    return duh @ V.T


@pytest.mark.parametrize("p", range(1, 8))
@pytest.mark.parametrize("a", [1.3, -0.7])
def test_fr_c0_equals_modal_dg_1d(p, a):
    rng = np.random.default_rng(p)
    K, h = 7, 0.37
    u = rng.standard_normal((K, p + 1))
    fr = residual_advection(u, a, h, p)
    dg = _modal_dg_residual(u, a, h, p)
    np.testing.assert_allclose(fr, dg, rtol=0, atol=1e-11 * np.abs(dg).max())
