"""L2 projection of a solution between orders (oracle; test infrastructure only).

The paper starts its cascade runs at low order and switches to a higher one; the state is carried
over by the L2 projection onto the new polynomial space (in reference coordinates, exact for the
DG-equivalent basis): modal coefficients of the source (Legendre products on the hexahedron, the
orthonormal triangle modes times Legendre on the prism), truncated or zero-padded to the target
degree, evaluated at the target's solution points.
"""
from __future__ import annotations

import numpy as np

from .basis import Basis1D
from .tri import Tri, modes, vandermonde


def line_transfer(p, q):
    """[q+1][p+1]: values at the order-q Gauss points of the projection of the order-p nodal
    polynomial through the Gauss points."""
    xp, xq = Basis1D(p).nodes, Basis1D(q).nodes
    Vp = np.polynomial.legendre.legvander(xp, p)
    Vq = np.polynomial.legendre.legvander(xq, q)
    m = min(p, q) + 1
    return Vq[:, :m] @ np.linalg.inv(Vp)[:m, :]


def tri_transfer(p, q):
    """[Nt_q][Nt_p] for the triangle: orthonormal modes of total degree <= min(p, q) kept."""
    Tp, Tq = Tri(p), Tri(q)
    mp, mq = modes(p), modes(q)
    keep = [k for k, (i, j) in enumerate(mp) if i + j <= q]
    cols = [mq.index(mp[k]) for k in keep]
    Vq = vandermonde(q, Tq.rs)
    return Vq[:, cols] @ np.linalg.inv(Tp.V)[keep, :]


def project(Qs, p, q):
    """[Q_hex [E][(p+1)^3][5], Q_prism [Ep][Nt_p (p+1)][5]] -> the same at order q."""
    L = line_transfer(p, q)
    H = np.kron(L, np.kron(L, L))
    out = [np.einsum('mn,env->emv', H, Qs[0])]
    P = np.kron(L, tri_transfer(p, q))
    out.append(np.einsum('mn,env->emv', P, Qs[1]))
    return out
