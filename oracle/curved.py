"""Quadratic (curved) element geometry for the mixed-element oracle (test infrastructure only).

Element maps: 27-node triquadratic hexahedra and 18-node quadratic prisms (node orders: corners,
edge midpoints, face centres, as listed in HEX27 / PRISM18 below); x(xi) and |J| from the shape
functions.  Metric terms S = |J| J^-1 (rows = reference directions) by the conservative curl form
of Kopriva (2006, "Metric identities and the discontinuous spectral element method on
curvilinear meshes"): with (n, m, l) cyclic,
    S[i][n] = -( curl_xi  I(X_l grad_xi X_m) )_i,
I the degree-p interpolant on a node set that contains the element's faces (Gauss-Lobatto
points on each hexahedron axis; the triangle's warp-and-blend nodes times Gauss-Lobatto points
in zeta on the prism).  S is then a polynomial of degree p evaluated exactly at any point, the
discrete metric identities sum_i D_i S[i][n] = 0 hold at the solution points, and a face's normal
depends only on the face's own geometry, so the two sides of an interface agree.  Here the
interpolant's derivatives are evaluated densely: 1D Lagrange product formulas along the line
directions, the triangle's nodal basis through its orthonormal modes.
"""
from __future__ import annotations

import numpy as np

from .tri import Tri, gauss_lobatto, grad_vandermonde, vandermonde

HEX27 = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1], [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1],
                  [0, -1, -1], [1, 0, -1], [0, 1, -1], [-1, 0, -1], [0, -1, 1], [1, 0, 1], [0, 1, 1], [-1, 0, 1],
                  [-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0],
                  [-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1], [0, 0, 0]], dtype=np.float64)
PRISM18 = np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1], [1, -1, 1], [-1, 1, 1],
                    [0, -1, -1], [0, 0, -1], [-1, 0, -1], [0, -1, 1], [0, 0, 1], [-1, 0, 1],
                    [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [0, -1, 0], [0, 0, 0], [-1, 0, 0]], dtype=np.float64)


def _quad1d(t, c):
    """Quadratic Lagrange function of the node c in {-1, 0, 1} and its derivative at t."""
    if c < 0:
        return t * (t - 1) / 2, t - 0.5
    if c > 0:
        return t * (t + 1) / 2, t + 0.5
    return 1 - t * t, -2 * t


def hex27_shape(ref):
    """N [M][27], dN [M][27][3] at reference points ref [M][3]."""
    M = ref.shape[0]
    N = np.ones((M, 27))
    dN = np.ones((M, 27, 3))
    for a, node in enumerate(HEX27):
        vals = [_quad1d(ref[:, d], node[d]) for d in range(3)]
        N[:, a] = vals[0][0] * vals[1][0] * vals[2][0]
        dN[:, a, 0] = vals[0][1] * vals[1][0] * vals[2][0]
        dN[:, a, 1] = vals[0][0] * vals[1][1] * vals[2][0]
        dN[:, a, 2] = vals[0][0] * vals[1][0] * vals[2][1]
    return N, dN


def prism18_shape(ref):
    """Quadratic triangle (corners lambda (2 lambda - 1), edge midpoints 4 lambda_i lambda_j) times
    the quadratic line in zeta."""
    r, s, z = ref[:, 0], ref[:, 1], ref[:, 2]
    lam = [-(r + s) / 2, (1 + r) / 2, (1 + s) / 2]
    dlam = [(-0.5, -0.5), (0.5, 0.0), (0.0, 0.5)]
    M = ref.shape[0]
    N = np.empty((M, 18))
    dN = np.empty((M, 18, 3))
    for a, node in enumerate(PRISM18):
        lb = np.array([-(node[0] + node[1]) / 2, (1 + node[0]) / 2, (1 + node[1]) / 2])
        ones = [i for i in range(3) if abs(lb[i] - 1) < 1e-12]
        if ones:                                  # corner i: lambda_i (2 lambda_i - 1)
            i = ones[0]
            T = lam[i] * (2 * lam[i] - 1)
            dT = [(4 * lam[i] - 1) * dlam[i][q] for q in range(2)]
        else:                                     # midpoint of edge (i, j): 4 lambda_i lambda_j
            i, j = [q for q in range(3) if abs(lb[q] - 0.5) < 1e-12]
            T = 4 * lam[i] * lam[j]
            dT = [4 * (dlam[i][q] * lam[j] + lam[i] * dlam[j][q]) for q in range(2)]
        Z, dZ = _quad1d(z, node[2])
        N[:, a] = T * Z
        dN[:, a, 0] = dT[0] * Z
        dN[:, a, 1] = dT[1] * Z
        dN[:, a, 2] = T * dZ
    return N, dN


def lagrange_1d(nodes, x):
    """Values [M][n] and derivatives [M][n] of the Lagrange polynomials of `nodes` at x (product
    formula)."""
    n = len(nodes)
    x = np.asarray(x, dtype=np.float64)
    L = np.ones((x.size, n))
    dL = np.zeros((x.size, n))
    for a in range(n):
        for b in range(n):
            if b != a:
                L[:, a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
        for c in range(n):
            if c == a:
                continue
            term = np.full(x.size, 1.0 / (nodes[a] - nodes[c]))
            for b in range(n):
                if b != a and b != c:
                    term *= (x - nodes[b]) / (nodes[a] - nodes[b])
            dL[:, a] += term
    return L, dL


def _hex_nodal(p, ref):
    """Nodal basis of the Gauss-Lobatto tensor nodes (index a + N b + N^2 c) and its three
    derivatives at ref."""
    g = gauss_lobatto(p)
    V = [lagrange_1d(g, ref[:, d]) for d in range(3)]
    N = p + 1
    idx = [(a, b, c) for c in range(N) for b in range(N) for a in range(N)]
    B = np.stack([V[0][0][:, a] * V[1][0][:, b] * V[2][0][:, c] for a, b, c in idx], 1)
    D = [np.stack([V[0][1][:, a] * V[1][0][:, b] * V[2][0][:, c] for a, b, c in idx], 1),
         np.stack([V[0][0][:, a] * V[1][1][:, b] * V[2][0][:, c] for a, b, c in idx], 1),
         np.stack([V[0][0][:, a] * V[1][0][:, b] * V[2][1][:, c] for a, b, c in idx], 1)]
    return B, D


def _prism_nodal(p, ref):
    """Nodal basis of (triangle warp-and-blend nodes) x (Gauss-Lobatto in zeta), index q + Nt k."""
    T = Tri(p)
    Lt = vandermonde(p, ref[:, :2]) @ T.Vinv
    Vr, Vs = grad_vandermonde(p, ref[:, :2])
    Lr, Ls = Vr @ T.Vinv, Vs @ T.Vinv
    Z, dZ = lagrange_1d(gauss_lobatto(p), ref[:, 2])
    cols = [(q, k) for k in range(p + 1) for q in range(T.Nt)]
    B = np.stack([Lt[:, q] * Z[:, k] for q, k in cols], 1)
    D = [np.stack([Lr[:, q] * Z[:, k] for q, k in cols], 1), np.stack([Ls[:, q] * Z[:, k] for q, k in cols], 1),
         np.stack([Lt[:, q] * dZ[:, k] for q, k in cols], 1)]
    return B, D


def interpolation_nodes(kind, p):
    """The face-containing node set of the curl form's interpolant."""
    g = gauss_lobatto(p) if p >= 1 else np.array([0.0])
    if kind == "hex":
        K, J, I_ = np.meshgrid(g, g, g, indexing="ij")
        return np.stack([I_.ravel(), J.ravel(), K.ravel()], 1)
    rs = Tri(p).rs
    return np.array([[rs[q, 0], rs[q, 1], g[k]] for k in range(p + 1) for q in range(rs.shape[0])])


def curved_geometry(kind, p):
    """geometry(X [E][nv][3], ref [M][3]) -> (x, |J|, S) for quadratic elements of `kind`."""
    shape = hex27_shape if kind == "hex" else prism18_shape
    nodal = _hex_nodal if kind == "hex" else _prism_nodal
    nodes = interpolation_nodes(kind, p)
    Nn, dNn = shape(nodes)

    def geometry(X, ref):
        N, dN = shape(ref)
        x = np.einsum('ma,eai->emi', N, X)
        J = np.einsum('mab,eai->emib', dN, X)                 # J[i][b] = dx_i / dxi_b
        detJ = np.linalg.det(J)
        Xn = np.einsum('ma,eai->emi', Nn, X)                  # positions at the interpolation nodes
        if p >= 2:
            # X_l measured from the element's corner centroid: for p >= 2 the interpolant reproduces
            # grad X_m (degree <= 2), so curl I(c grad X_m) = 0 and S is unchanged; the shift only
            # removes the cancellation of coordinates large against the element size.
            nc = 8 if kind == "hex" else 6
            Xn = Xn - X[:, :nc, :].mean(axis=1)[:, None, :]
        Jn = np.einsum('mab,eai->emib', dNn, X)               # gradients there
        _, Lag_d = nodal(p, ref)                              # derivatives of the nodal interpolant
        S = np.empty(x.shape[:2] + (3, 3))
        for n in range(3):
            m, l = (n + 1) % 3, (n + 2) % 3
            v = Xn[:, :, l, None] * Jn[:, :, m, :]            # v[e][node][k] = X_l d_k X_m
            for i in range(3):
                j, k = (i + 1) % 3, (i + 2) % 3
                S[:, :, i, n] = -(np.einsum('mq,eq->em', Lag_d[j], v[:, :, k])
                                  - np.einsum('mq,eq->em', Lag_d[k], v[:, :, j]))
        return x, detJ, S
    return geometry
