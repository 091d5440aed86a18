"""1D FR for linear advection u_t + a u_x = 0 on a periodic uniform mesh (oracle; test infrastructure).

It uses the same 1D building blocks as the hexahedral oracle (Gauss-Legendre points, Lagrange
derivative matrix, boundary values, correction derivative) and exists to pin them: with the
correction g = right/left Radau polynomials the FR scheme reproduces nodal collocated DG (section
"FR Algorithm" of arXiv 2308.06605, citing Huynh 2007), which the tests compare against an
independent modal Legendre DG discretisation.

Per element of width h (|J| = h/2):
  du/dxi-residual = -(2/h) [ D f + g_R'(xi) (f^I_R - f(+1)) + g_R'(-xi) (f^I_Lperp - f_Lperp) ],
where on the left face the outward normal is -1 so f_Lperp = -f(-1) and f^I_Lperp = -f^I_L.
The common flux is the upwind flux a u^- (a > 0: the left neighbour's trace).
"""
from __future__ import annotations

import numpy as np

from .basis import Basis1D


def residual_advection(u, a: float, h: float, p: int, c: float = 0.0):
    """u: [K][N] nodal values per element (K elements, periodic).  Returns du/dt [K][N].
    c selects the correction function of the energy-stable family (basis.correction_right)."""
    b = Basis1D(p, c)
    f = a * u
    uL = u @ b.l_minus                      # trace at xi = -1 of each element
    uR = u @ b.l_plus                       # trace at xi = +1
    fR_own = f @ b.l_plus
    fL_own = f @ b.l_minus
    if a >= 0:
        fI_right = a * uR                   # interface e | e+1 takes element e's right trace
        fI_left = a * np.roll(uR, 1)        # interface e-1 | e
    else:
        fI_right = a * np.roll(uL, -1)
        fI_left = a * uL
    div = f @ b.D.T
    corr = (np.outer(fI_right - fR_own, b.h_plus)
            + np.outer((-fI_left) - (-fL_own), b.h_minus))
    return -(2.0 / h) * (div + corr)
