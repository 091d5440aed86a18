"""Independent 40-digit restatement of the hexahedral Navier-Stokes residual on small periodic
lattices (oracle; test infrastructure only: only tests/ and the golden-file scripts beside them
use it).

Nodal DG in WEAK form with the exact (non-lumped) mass matrix and over-integrated quadrature, at
40 significant digits (mpmath), on 1..n1 affine elements stacked along the first lattice axis and
periodic in all directions.  With the c = 0 correction the FR scheme of arXiv 2308.06605 (section
"FR Algorithm", Eq. 3) equals this strong/weak-form DG with collocated fluxes:
    M dQ/dt = int grad(phi) . H^delta dx - sum_faces int phi (H^I . n)^delta dS,
with the BR2 gradient  M G = int phi grad Q^delta + sum_f int phi dQ^delta n dS  and the face
lifting  M r_f = int_f phi dQ^delta n dS  (Rusanov inviscid flux, the average of the two sides'
face gradients as the common gradient).  Nothing here uses the FP64 oracle's basis, operators,
connectivity or gas functions, so the two pin each other.
"""
import itertools
from fractions import Fraction

import mpmath
import numpy as np

mp = mpmath.mp


def _gl_mp(N):
    """Gauss-Legendre nodes/weights at mp precision (roots of P_N polished by findroot)."""
    guess, _ = np.polynomial.legendre.leggauss(N)
    xs, ws = [], []
    for g in guess:
        x = mp.findroot(lambda t: mp.legendre(N, t), mp.mpf(g))
        dP = mp.diff(lambda t: mp.legendre(N, t), x)
        xs.append(x)
        ws.append(2 / ((1 - x * x) * dP * dP))
    return xs, ws


def _lag(nodes, j, x):
    v = mp.mpf(1)
    for m, xm in enumerate(nodes):
        if m != j:
            v *= (x - xm) / (nodes[j] - xm)
    return v


def _dlag(nodes, j, x):
    s = mp.mpf(0)
    for k in range(len(nodes)):
        if k == j:
            continue
        t = 1 / (nodes[j] - nodes[k])
        for m in range(len(nodes)):
            if m != j and m != k:
                t *= (x - nodes[m]) / (nodes[j] - nodes[m])
        s += t
    return s


def _prim(q, gam):
    rho = q[0]
    u = [q[1] / rho, q[2] / rho, q[3] / rho]
    p = (gam - 1) * (q[4] - rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2) / 2)
    return rho, u, p


def _flux_inv(q, gam):
    rho, u, p = _prim(q, gam)
    return [[rho * u[j]] + [rho * u[i] * u[j] + (p if i == j else 0) for i in range(3)]
            + [(q[4] + p) * u[j]] for j in range(3)]


def _flux_visc(q, g, gam, R, mu, Pr):
    """g[j][v] = dQ_v/dx_j."""
    rho, u, p = _prim(q, gam)
    E = q[4]
    du = [[(g[j][1 + i] - u[i] * g[j][0]) / rho for j in range(3)] for i in range(3)]
    T_grad = [(gam - 1) / R * ((g[j][4] - E / rho * g[j][0]) / rho - sum(u[i] * du[i][j] for i in range(3)))
              for j in range(3)]
    div = du[0][0] + du[1][1] + du[2][2]
    tau = [[mu * (du[i][j] + du[j][i] - (mp.mpf(2) / 3 * div if i == j else 0)) for j in range(3)] for i in range(3)]
    k = mu * gam * R / ((gam - 1) * Pr)
    return [[0] + [tau[i][j] for i in range(3)] + [sum(u[i] * tau[i][j] for i in range(3)) + k * T_grad[j]]
            for j in range(3)]


def _rusanov(qa, qb, n, gam):
    Fa, Fb = _flux_inv(qa, gam), _flux_inv(qb, gam)
    nm = mp.sqrt(n[0] ** 2 + n[1] ** 2 + n[2] ** 2)
    lam = []
    for q in (qa, qb):
        rho, u, p = _prim(q, gam)
        lam.append(abs(sum(u[j] * n[j] for j in range(3))) / nm + mp.sqrt(gam * p / rho))
    L = max(lam)
    return [sum((Fa[j][v] + Fb[j][v]) * n[j] for j in range(3)) / 2 - L * nm * (qb[v] - qa[v]) / 2 for v in range(5)]


def _exact(x):
    """A constant at the working precision: Fractions and ints exactly, floats by their binary value,
    strings as decimal numbers (e.g. "1.4" is 1.4 to 40 digits, not its nearest double)."""
    if isinstance(x, Fraction):
        return mp.mpf(x.numerator) / x.denominator
    return mp.mpf(x)


def brute_force_residual(Q, p, n1, Amat, hbox, gam, R, mu, Pr, eta, viscous):
    """Residual (float64, rounded from 40 digits) of n1 elements stacked along the first lattice
    axis of the affine map x = Amat diag(hbox) xi, periodic in all directions; Q [n1][N^3][5] in the
    canonical point order; gam, R, mu, Pr, eta as Fractions, ints, floats or decimal strings,
    converted at 40 digits; BR2 viscous terms if viscous."""
    mp.dps = 40
    gam, R, mu, Pr, eta = (_exact(v) for v in (gam, R, mu, Pr, eta))
    N = p + 1
    nodes, _ = _gl_mp(N)
    xq, wq = _gl_mp(N + 2)
    M1 = len(xq)
    J = mpmath.matrix(3, 3)
    for i in range(3):
        for b in range(3):
            J[i, b] = mp.mpf(Amat[i][b]) * mp.mpf(hbox[b]) / 2
    detJ = mpmath.det(J)
    Jinv = J ** -1
    Lq = [[_lag(nodes, i, x) for i in range(N)] for x in xq]          # l_i(xq_a)
    dLq = [[_dlag(nodes, i, x) for i in range(N)] for x in xq]
    Lb = {s: [_lag(nodes, i, mp.mpf(s)) for i in range(N)] for s in (-1, 1)}
    Ln = [[_lag(nodes, i, x) for i in range(N)] for x in nodes]      # identity, kept explicit
    dLn = [[_dlag(nodes, i, x) for i in range(N)] for x in nodes]
    m1 = [[sum(wq[a] * Lq[a][i] * Lq[a][j] for a in range(M1)) for j in range(N)] for i in range(N)]
    m1inv = mpmath.matrix(m1) ** -1
    pts = [(m % N, (m // N) % N, m // (N * N)) for m in range(N ** 3)]   # (i, j, k) of canonical m
    idx = {t: t[0] + N * t[1] + N * N * t[2] for t in pts}
    Qm = [[[mp.mpf(float(Q[e, m, v])) for v in range(5)] for m in range(N ** 3)] for e in range(n1)]

    def minv_apply(rhs):
        """Apply (|J| m1 x m1 x m1)^-1 to rhs[m][...] (tensor solve)."""
        out = [[mp.mpf(0)] * len(rhs[0]) for _ in range(N ** 3)]
        for (i, j, k) in pts:
            for (a, b, c) in pts:
                f = m1inv[i, a] * m1inv[j, b] * m1inv[k, c]
                if f != 0:
                    src, dst = rhs[idx[(a, b, c)]], out[idx[(i, j, k)]]
                    for v in range(len(src)):
                        dst[v] += f * src[v]
        return [[x / detJ for x in row] for row in out]

    faces = [(d, s) for d in range(3) for s in (-1, 1)]

    def face_ref(d, s, t1, t2):
        r = [None, None, None]
        tang = [a for a in range(3) if a != d]
        r[d] = s
        r[tang[0]], r[tang[1]] = t1, t2
        return r

    def nscaled(d, s):
        return [s * detJ * Jinv[d, j] for j in range(3)]

    def eval_nodal(vals, r):
        """Interpolant of nodal values vals[m][...] at reference point r."""
        li = [[_lag(nodes, i, r[a]) for i in range(N)] for a in range(3)]
        out = [mp.mpf(0)] * len(vals[0])
        for (i, j, k) in pts:
            w = li[0][i] * li[1][j] * li[2][k]
            if w != 0:
                for v in range(len(out)):
                    out[v] += w * vals[idx[(i, j, k)]][v]
        return out

    def nbr(e, d, s):
        return ((e + s) % n1) if d == 0 else e

    # Traces at the flux points of each face (GL points of the face).
    fp = list(itertools.product(range(N), repeat=2))
    trace = {}
    for e in range(n1):
        for (d, s) in faces:
            trace[(e, d, s)] = [eval_nodal(Qm[e], face_ref(d, s, nodes[a], nodes[b])) for (a, b) in fp]
    jump = {}
    for e in range(n1):
        for (d, s) in faces:
            other = trace[(nbr(e, d, s), d, -s)]
            own = trace[(e, d, s)]
            jump[(e, d, s)] = [[(other[q][v] - own[q][v]) / 2 for v in range(5)] for q in range(len(fp))]

    def face_integral(e, d, s, fvals, ncomp):
        """int_face phi_m f^delta dxi_t, f given at the face GL points, over-integrated."""
        out = [[mp.mpf(0)] * ncomp for _ in range(N ** 3)]
        tang = [a for a in range(3) if a != d]
        for a1 in range(M1):
            for a2 in range(M1):
                w = wq[a1] * wq[a2]
                lf = [Lq[a1][a] * Lq[a2][b] for (a, b) in fp]          # face interpolant weights
                fv = [sum(lf[q] * fvals[q][c] for q in range(len(fp))) for c in range(ncomp)]
                for (i, j, k) in pts:
                    ijk = (i, j, k)
                    phi = Lb[s][ijk[d]] * Lq[a1][ijk[tang[0]]] * Lq[a2][ijk[tang[1]]]
                    if phi != 0:
                        row = out[idx[ijk]]
                        for c in range(ncomp):
                            row[c] += w * phi * fv[c]
        return out

    # Gradients (BR2): corrected volume gradient and per-face lifts.
    grads, gfaces = {}, {}
    if viscous:
        for e in range(n1):
            gref = []                                                   # reference gradient of Q^delta at nodes
            for (i, j, k) in pts:
                g = [[mp.mpf(0)] * 5 for _ in range(3)]
                for a in range(N):
                    for v in range(5):
                        g[0][v] += dLn[i][a] * Qm[e][idx[(a, j, k)]][v]
                        g[1][v] += dLn[j][a] * Qm[e][idx[(i, a, k)]][v]
                        g[2][v] += dLn[k][a] * Qm[e][idx[(i, j, a)]][v]
                gref.append(g)
            gunc = [[[sum(Jinv[d, jj] * gref[m][d][v] for d in range(3)) for v in range(5)] for jj in range(3)]
                    for m in range(N ** 3)]
            lifts = {}
            total = [[gunc[m][jj][v] for jj in range(3) for v in range(5)] for m in range(N ** 3)]
            for (d, s) in faces:
                n = nscaled(d, s)
                fv = [[jump[(e, d, s)][q][v] * n[jj] for jj in range(3) for v in range(5)] for q in range(len(fp))]
                rf = minv_apply(face_integral(e, d, s, fv, 15))
                lifts[(d, s)] = rf
                for m in range(N ** 3):
                    for c in range(15):
                        total[m][c] += rf[m][c]
            grads[e] = [[[total[m][jj * 5 + v] for v in range(5)] for jj in range(3)] for m in range(N ** 3)]
            for (d, s) in faces:
                rf = lifts[(d, s)]
                vals = [[gunc[m][jj][v] + eta * rf[m][jj * 5 + v] for jj in range(3) for v in range(5)]
                        for m in range(N ** 3)]
                gfaces[(e, d, s)] = [eval_nodal(vals, face_ref(d, s, nodes[a], nodes[b])) for (a, b) in fp]
    out = np.zeros((n1, N ** 3, 5))
    for e in range(n1):
        H = []
        for m in range(N ** 3):
            F = _flux_inv(Qm[e][m], gam)
            if viscous:
                Fv = _flux_visc(Qm[e][m], grads[e][m], gam, R, mu, Pr)
                F = [[F[j][v] - Fv[j][v] for v in range(5)] for j in range(3)]
            H.append(F)
        rhs = [[mp.mpf(0)] * 5 for _ in range(N ** 3)]
        # Volume term int grad_x(phi_m) . H^delta dx = |J| int (J^-T grad_xi phi)_j H_j dxi.
        for a in range(M1):
            for b in range(M1):
                for c in range(M1):
                    w = wq[a] * wq[b] * wq[c] * detJ
                    lw = [Lq[a][i] * Lq[b][j] * Lq[c][k] for (i, j, k) in pts]
                    Hq = [[sum(lw[m] * H[m][jj][v] for m in range(N ** 3)) for v in range(5)] for jj in range(3)]
                    for (i, j, k) in pts:
                        gxi = [dLq[a][i] * Lq[b][j] * Lq[c][k], Lq[a][i] * dLq[b][j] * Lq[c][k],
                               Lq[a][i] * Lq[b][j] * dLq[c][k]]
                        gx = [sum(Jinv[d, jj] * gxi[d] for d in range(3)) for jj in range(3)]
                        row = rhs[idx[(i, j, k)]]
                        for v in range(5):
                            row[v] += w * sum(gx[jj] * Hq[jj][v] for jj in range(3))
        for (d, s) in faces:
            n = nscaled(d, s)
            own = trace[(e, d, s)]
            oth = trace[(nbr(e, d, s), d, -s)]
            fvals = []
            for q in range(len(fp)):
                fI = _rusanov(own[q], oth[q], n, gam)
                if viscous:
                    go = gfaces[(e, d, s)][q]
                    gn = gfaces[(nbr(e, d, s), d, -s)][q]
                    gc = [[(go[jj * 5 + v] + gn[jj * 5 + v]) / 2 for v in range(5)] for jj in range(3)]
                    qc = [(own[q][v] + oth[q][v]) / 2 for v in range(5)]
                    Fv = _flux_visc(qc, gc, gam, R, mu, Pr)
                    fI = [fI[v] - sum(Fv[jj][v] * n[jj] for jj in range(3)) for v in range(5)]
                fvals.append(fI)
            sf = face_integral(e, d, s, fvals, 5)
            for m in range(N ** 3):
                for v in range(5):
                    rhs[m][v] -= sf[m][v]
        dq = minv_apply(rhs)
        out[e] = np.array([[float(x) for x in row] for row in dq])
    return out
