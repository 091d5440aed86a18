"""Hexahedral FR residual for the compressible Navier-Stokes equations (oracle; test infrastructure only).

Follows the section "FR Algorithm" of arXiv 2308.06605 step by step, in plain FP64 with dense
per-element operators built as Kronecker products of the 1D arrays of `basis`:

  Eq. 1   Q^ = |J| Q, F^_d = sum_j S_dj F_j with S = |J| J^-1 (J_ij = dx_i/dxi_j), from the
          trilinear map of each hexahedron.
  Eq. 2   nodal Lagrange interpolants on the N^3 tensor Gauss-Legendre points; point index
          m = i + N j + N^2 k (i along xi, j along eta, k along zeta).
  Eq. 3   dQ/dt = -|J|^-1 [ sum_d D_d F^_d + sum_faces C_f (F^I_perp - F_perp) ] + S, where
          F_perp is the interpolated transformed flux dotted with the outward reference normal,
          F^I_perp the common normal flux (Rusanov) times the area-scaled physical normal, and
          C_f the divergence of the face's correction field: along the face's normal line it
          takes the values g_R'(s xi_i) (s = outward sign); g is the DG-equivalent Radau
          polynomial (the paper's choice) or, with phys.vcjh_c = c != 0, the member c of the
          energy-stable family of Vincent, Castonguay & Jameson (basis.correction_right).  The
          same correction fields correct the gradient (viscous part).
  Viscous part (BR2; the paper uses LDG, this build's reading takes BR2): the common solution
  Q^I = (Q- + Q+)/2 corrects the reference gradient with the same correction fields,
  grad_x Q = J^-T grad_xi Q; at each face the side gradient is the uncorrected gradient
  interpolated to the face plus eta times the face's own lifting r_f interpolated to the face;
  the common gradient is the average of the two sides; the common viscous flux is
  F_v(Q^I, common gradient) . n.
  Viscous part, LDG (viscous = 2): per interface the side whose face normal points along
  gas.LDG_SWITCH supplies Q^I (its own trace), the other side supplies the common gradient; side
  gradients are the corrected gradient interpolated to the face; the common flux adds the penalty
  tau |n| (Q_0 - Q_1) (side 0's frame) and at boundaries tau |n| (Q- - Q_b).
  Time: classical four-stage Runge-Kutta.

Reference faces: f = 2 d + (s + 1)/2, i.e. 0: xi=-1, 1: xi=+1, 2: eta=-1, 3: eta=+1,
4: zeta=-1, 5: zeta=+1.  Flux points of face f are ordered by the two remaining axes with the
lower axis fastest.

Connectivity is found geometrically: faces are paired by their (periodically shifted)
centroids, flux points by their physical coordinates.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from . import gas
from . import mlp
from .basis import Basis1D

FACE_AXIS = (0, 0, 1, 1, 2, 2)
FACE_SIGN = (-1, 1, -1, 1, -1, 1)
HEX_REF_VERTS = np.array([
    [-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
    [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.float64)

BC_WALL_ISOTHERMAL = 1
BC_CHAR_INFLOW = 2
BC_CHAR_OUTFLOW = 3
BC_DIRICHLET = 4
PR_TURB = 0.9      # turbulent Prandtl number of the eddy-viscosity closure


def trilinear_geometry(X, ref):
    """Physical points, Jacobian determinant and S = |J| J^-1 of trilinear hexahedra.

    X: [E][8][3] vertex coordinates, ref: [M][3] reference points.  Shape functions
    N_v = prod_a (1 + c_va xi_a)/2 with c_v the reference vertex coordinates.
    Returns x [E][M][3], detJ [E][M], S [E][M][3][3] with S[d][j] = |J| (J^-1)_dj.
    """
    c = HEX_REF_VERTS
    fac = (1.0 + ref[:, None, :] * c[None, :, :]) / 2.0          # [M][8][3]
    Nv = np.prod(fac, axis=2)                                    # [M][8]
    dN = np.empty(ref.shape[:1] + (8, 3))                        # dN_v/dxi_b
    for b in range(3):
        others = [a for a in range(3) if a != b]
        dN[:, :, b] = (c[None, :, b] / 2.0) * fac[:, :, others[0]] * fac[:, :, others[1]]
    x = np.einsum('mv,evi->emi', Nv, X)
    J = np.einsum('mvb,evi->emib', dN, X)                        # J[i][b] = dx_i/dxi_b
    detJ = np.linalg.det(J)
    S = detJ[..., None, None] * np.linalg.inv(J)
    return x, detJ, S


def boundary_states(kind, prm, Qm, n, g, Rg):
    """Boundary face of kind `kind` with parameters `prm`: (ghost state for the Riemann flux,
    common solution Q^I) at its flux points, from the interior trace Qm [Nf][5] and the outward
    area-scaled normal n [Nf][3] (gas constants g = gamma, Rg = R).

    The paper lists boundary conditions among its physical models without stating them;
    this build's readings are:
      wall (isothermal no-slip, T_w): ghost = interior density and energy with reversed
        momentum (the mirror state); Q^I = wall state (interior density, zero velocity,
        T = T_w).
      Dirichlet (exterior state Q_b): ghost = Q^I = Q_b.
      characteristic outflow (static p_b): interior entropy, tangential velocity and the
        outgoing invariant u.n^ + 2c/(gamma-1); ghost = Q^I = that boundary state.
      characteristic inflow (total p0, total T0, unit direction d): interior outgoing
        invariant; speed V from (d.n^)V + 2c_b/(gamma-1) = invariant with
        c_b^2 = gamma R (T0 - V^2/(2 cp)); static state from the isentropic relations;
        ghost = Q^I = that state.
    """
    rho, u, p = gas.primitives(Qm, g)
    if kind == BC_DIRICHLET:
        Qb = np.broadcast_to(prm[:5], Qm.shape).copy()
        return Qb, Qb
    if kind == BC_WALL_ISOTHERMAL:
        ghost = Qm.copy()
        ghost[..., 1:4] *= -1.0
        Qi = np.zeros_like(Qm)
        Qi[..., 0] = rho
        Qi[..., 4] = rho * Rg * prm[0] / (g - 1.0)
        return ghost, Qi
    nh = n / np.linalg.norm(n, axis=-1, keepdims=True)
    un = np.sum(u * nh, axis=-1)
    c = np.sqrt(g * p / rho)
    Rplus = un + 2.0 * c / (g - 1.0)
    if kind == BC_CHAR_OUTFLOW:
        pb = prm[0]
        s_ent = p / rho ** g
        rb = (pb / s_ent) ** (1.0 / g)
        cb = np.sqrt(g * pb / rb)
        unb = Rplus - 2.0 * cb / (g - 1.0)
        ub = u + (unb - un)[..., None] * nh
        Qb = np.stack([rb, rb * ub[..., 0], rb * ub[..., 1], rb * ub[..., 2],
                       pb / (g - 1.0) + 0.5 * rb * np.sum(ub * ub, axis=-1)], axis=-1)
        return Qb, Qb
    if kind == BC_CHAR_INFLOW:
        p0, T0 = prm[0], prm[1]
        d = np.asarray(prm[2:5], dtype=np.float64)
        d = d / np.linalg.norm(d)
        a = nh @ d
        A = a * a + 2.0 / (g - 1.0)
        B = -2.0 * a * Rplus
        Cc = Rplus * Rplus - (2.0 / (g - 1.0)) ** 2 * g * Rg * T0
        V = (-B + np.sqrt(B * B - 4.0 * A * Cc)) / (2.0 * A)
        cp = g * Rg / (g - 1.0)
        Tb = T0 - V * V / (2.0 * cp)
        pb = p0 * (Tb / T0) ** (g / (g - 1.0))
        rb = pb / (Rg * Tb)
        ub = V[..., None] * d
        Qb = np.stack([rb, rb * ub[..., 0], rb * ub[..., 1], rb * ub[..., 2],
                       pb / (g - 1.0) + 0.5 * rb * V * V], axis=-1)
        return Qb, Qb
    raise ValueError("unknown boundary kind %d" % kind)


class HexFR:
    """Oracle FR discretisation of one hexahedral mesh at uniform order p."""

    def __init__(self, desc, phys, p: int):
        self.phys = phys
        self.p = p
        self.b = b = Basis1D(p, getattr(phys, "vcjh_c", 0.0))
        self.N = N = p + 1
        self.Np = N ** 3
        self.Nf = N * N
        I = np.eye(N)
        D = b.D
        self.Dop = [np.kron(I, np.kron(I, D)), np.kron(I, np.kron(D, I)), np.kron(D, np.kron(I, I))]
        self.Lf, self.Cf = [], []
        for f in range(6):
            d, s = FACE_AXIS[f], FACE_SIGN[f]
            row = (b.l_plus if s > 0 else b.l_minus)[None, :]
            col = (b.h_plus if s > 0 else b.h_minus)[:, None]
            if d == 0:
                self.Lf.append(np.kron(I, np.kron(I, row)))
                self.Cf.append(np.kron(I, np.kron(I, col)))
            elif d == 1:
                self.Lf.append(np.kron(I, np.kron(row, I)))
                self.Cf.append(np.kron(I, np.kron(col, I)))
            else:
                self.Lf.append(np.kron(row, np.kron(I, I)))
                self.Cf.append(np.kron(col, np.kron(I, I)))
        xi = b.nodes
        K, Jj, Ii = np.meshgrid(xi, xi, xi, indexing="ij")        # [k][j][i]
        self.ref_sol = np.stack([Ii.ravel(), Jj.ravel(), K.ravel()], axis=1)
        self.ref_face = []
        for f in range(6):
            d, s = FACE_AXIS[f], FACE_SIGN[f]
            A, B = np.meshgrid(xi, xi, indexing="ij")             # [slow][fast]
            pts = np.zeros((self.Nf, 3))
            tang = [a for a in range(3) if a != d]
            pts[:, tang[0]] = B.ravel()
            pts[:, tang[1]] = A.ravel()
            pts[:, d] = s
            self.ref_face.append(pts)
        self._geometry(desc)
        self._connect(desc)
        self.closure = None

    def set_closure(self, params, scales):
        """Enable the eddy-viscosity closure (oracle.mlp): per element nu_t from the element-mean
        corrected velocity gradient; mu -> mu + rho nu_t, kappa -> kappa + rho nu_t cp / Pr_t in the
        volume flux, and with the average of the two elements' nu_t at interfaces."""
        self.closure = (np.asarray(params, dtype=np.float64), scales)

    def _closure_nu(self, Q, grad):
        rho = Q[..., 0]
        u = Q[..., 1:4] / rho[..., None]
        gu = (grad[..., :, 1:4] - grad[..., :, 0:1] * u[..., None, :]) / rho[..., None, None]   # [e][m][j][i]
        gu = np.swapaxes(gu, -1, -2)                                                            # du_i/dx_j
        wJ = self.W[None, :] * self.detJ
        mean = np.einsum('em,emij->eij', wJ, gu) / wJ.sum(axis=1)[:, None, None]
        X = mlp.features(mean, self.h, self.p)
        return mlp.eddy_viscosity(self.closure[0], self.closure[1], X)

    # ------------------------------------------------------------------ geometry (Eq. 1)
    def _geometry(self, desc):
        X = desc.xyz[desc.hex]
        self.E = X.shape[0]
        self.x, self.detJ, self.S = trilinear_geometry(X, self.ref_sol)
        if np.any(self.detJ <= 0):
            raise ValueError("non-positive Jacobian")
        self.xf = np.empty((self.E, 6, self.Nf, 3))
        self.nf = np.empty((self.E, 6, self.Nf, 3))                # area-scaled outward normal
        for f in range(6):
            xf, _, Sf = trilinear_geometry(X, self.ref_face[f])
            self.xf[:, f] = xf
            self.nf[:, f] = FACE_SIGN[f] * Sf[:, :, FACE_AXIS[f], :]
        w = self.b.weights
        W = np.kron(w, np.kron(w, w))                             # quadrature weights at m
        self.W = W
        self.vol = np.sum(W[None, :] * self.detJ, axis=1)
        self.h = self.vol ** (1.0 / 3.0)

    # ------------------------------------------------------------------ connectivity
    def _connect(self, desc):
        E, N = self.E, self.N
        corner_ids = [np.where(HEX_REF_VERTS[:, FACE_AXIS[f]] == FACE_SIGN[f])[0] for f in range(6)]
        btag = {tuple(sorted(nodes)): int(t) for nodes, t in zip(desc.bface_nodes.tolist(), desc.bface_tag.tolist())}
        shift_of_tag = {}
        for per in desc.periodic:
            shift_of_tag[per.tag_b] = np.asarray(per.t, dtype=np.float64)
            shift_of_tag.setdefault(per.tag_a, np.zeros(3))
        bc_of_tag = {bc.tag: bc for bc in desc.bcs}
        cent = np.empty((E * 6, 3))
        shift = np.zeros((E * 6, 3))
        face_tag = np.zeros(E * 6, dtype=np.int64)
        for e in range(E):
            for f in range(6):
                nodes = desc.hex[e, corner_ids[f]]
                cent[6 * e + f] = desc.xyz[nodes].mean(axis=0)
                face_tag[6 * e + f] = btag.get(tuple(sorted(nodes.tolist())), 0)
        bc_faces = []
        pairable = np.ones(E * 6, dtype=bool)
        for g in range(E * 6):
            t = face_tag[g]
            if t == 0:
                continue
            if t in shift_of_tag:
                shift[g] = shift_of_tag[t]
            elif t in bc_of_tag:
                bc_faces.append(g)
                pairable[g] = False
            else:
                raise ValueError(f"boundary tag {t} has no boundary condition")
        idx = np.where(pairable)[0]
        key = cent[idx] - shift[idx]
        hmin = float(np.min(self.h))
        tree = cKDTree(key)
        pairs = np.array(sorted(tree.query_pairs(r=1e-6 * hmin)), dtype=np.int64).reshape(-1, 2)
        if len(pairs) * 2 != len(idx) or len(np.unique(pairs)) != len(idx):
            raise ValueError("unmatched or multiply matched faces")
        gL, gR = idx[pairs[:, 0]], idx[pairs[:, 1]]
        self.eL, self.fL = gL // 6, gL % 6
        self.eR, self.fR = gR // 6, gR % 6
        xL = self.xf[self.eL, self.fL] - shift[gL][:, None, :]
        xR = self.xf[self.eR, self.fR] - shift[gR][:, None, :]
        dist = np.linalg.norm(xL[:, :, None, :] - xR[:, None, :, :], axis=-1)
        self.perm = np.argmin(dist, axis=2)                       # R fpt matching L fpt q
        if np.max(np.min(dist, axis=2)) > 1e-6 * hmin:
            raise ValueError("flux points do not match across an interface")
        self.invperm = np.argsort(self.perm, axis=1)
        P = len(gL)
        self.n_if = P
        rows = np.arange(P)[:, None]
        self.nL = self.nf[self.eL, self.fL]
        self.nR_matched = self.nf[self.eR, self.fR][rows, self.perm]
        bc_faces = np.array(bc_faces, dtype=np.int64)
        self.bE, self.bF = bc_faces // 6, bc_faces % 6
        self.b_kind = np.array([bc_of_tag[face_tag[g]].kind for g in bc_faces], dtype=np.int64)
        self.b_params = [np.asarray(bc_of_tag[face_tag[g]].params, dtype=np.float64) for g in bc_faces]

    # ------------------------------------------------------------------ helpers
    def solution_points(self):
        """Physical coordinates of the solution points, [E][N^3][3] in canonical order."""
        return self.x.copy()

    def _interp_faces(self, A):
        """A [E][Np][...] -> [E][6][Nf][...] values at the flux points of each face."""
        return np.stack([np.einsum('qm,em...->eq...', self.Lf[f], A) for f in range(6)], axis=1)

    def _lift(self, f, B):
        """C_f applied to face data B [E][Nf][...] -> [E][Np][...]."""
        return np.einsum('mq,eq...->em...', self.Cf[f], B)

    def _boundary_states(self, Qm, n, k):
        """Boundary face k: (ghost, Q^I) by `boundary_states`."""
        return boundary_states(self.b_kind[k], self.b_params[k], Qm, n, self.phys.gamma, self.phys.R)

    # ------------------------------------------------------------------ residual (Eq. 3)
    def residual(self, Q, t=0.0, magnitude=False):
        """dQ/dt at the solution points; Q and the result are [E][N^3][5].

        With magnitude=True it returns instead the entrywise magnitude of the final sum,
        |J|^-1 [sum_d |D_d| |F^_d| + sum_f |C_f| (|F^I_perp| + |L_f| |F^_d|)], the natural scale of
        the rounding error of any evaluation order of Eq. 3 (used for tolerances).
        """
        ph = self.phys
        gam = ph.gamma
        viscous = ph.viscous != 0 and ph.mu != 0.0
        ldg = viscous and ph.viscous == 2
        E, Nf = self.E, self.Nf
        rows = np.arange(self.n_if)[:, None]
        # Solution at flux points, both sides of every interface.
        Qf = self._interp_faces(Q)                                 # [E][6][Nf][5]
        QL = Qf[self.eL, self.fL]
        QR = Qf[self.eR, self.fR][rows, self.perm]
        Qc_face = np.empty_like(Qf)                                # common solution per element face
        if ldg:
            up = (self.nL.sum(axis=1) @ gas.LDG_SWITCH) > 0        # side 0 supplies Q^I
            QI = np.where(up[:, None, None], QL, QR)
        else:
            QI = 0.5 * (QL + QR)
        Qc_face[self.eL, self.fL] = QI
        Qc_face[self.eR, self.fR] = QI[rows, self.invperm]
        ghosts, bstates = [], []
        for k in range(len(self.bE)):
            Qm = Qf[self.bE[k], self.bF[k]]
            Qg, Qb = self._boundary_states(Qm, self.nf[self.bE[k], self.bF[k]], k)
            ghosts.append(Qg)
            bstates.append(Qb)
            Qc_face[self.bE[k], self.bF[k]] = Qb
        dQ = Qc_face - Qf                                          # Q^I - Q- per element face
        Sinv = self.S / self.detJ[..., None, None]                 # J^-1, [E][Np][d][j]
        if viscous:
            # Reference gradients: uncorrected D_d Q, corrected adds sum_f s_f C_f dQ_f on axis d_f.
            g_unc = np.stack([np.einsum('mn,env->emv', self.Dop[d], Q) for d in range(3)], axis=2)  # [E][Np][d][5]
            g_cor = g_unc.copy()
            lifts = []
            for f in range(6):
                lf = FACE_SIGN[f] * self._lift(f, dQ[:, f])        # [E][Np][5]
                g_cor[:, :, FACE_AXIS[f], :] += lf
                lifts.append(lf)
            grad = np.einsum('emdj,emdv->emjv', Sinv, g_cor)       # physical, corrected
            grad_unc = np.einsum('emdj,emdv->emjv', Sinv, g_unc)
            # Face gradient per side: interpolated uncorrected gradient + eta * own lift r_f.
            gface = np.empty((E, 6, Nf, 3, 5))
            for f in range(6):
                r_f = np.einsum('emj,emv->emjv', Sinv[:, :, FACE_AXIS[f], :], lifts[f])
                if ldg:
                    gface[:, f] = np.einsum('qm,emjv->eqjv', self.Lf[f], grad)
                else:
                    gface[:, f] = np.einsum('qm,emjv->eqjv', self.Lf[f], grad_unc + ph.br2_eta * r_f)
            kappa0 = ph.mu * gam * ph.R / ((gam - 1.0) * ph.Pr)
            cp = gam * ph.R / (gam - 1.0)
            nu_el = np.zeros(E)
            if self.closure is not None:
                nu_el = self._closure_nu(Q, grad)
            self.last_nu = nu_el
            rho_v = Q[..., 0]
            Fv = gas.viscous_flux(Q, grad, gam, ph.R, ph.mu + rho_v * nu_el[:, None], ph.Pr,
                                  kappa=kappa0 + rho_v * nu_el[:, None] * cp / PR_TURB)
        # Physical and transformed flux at solution points.
        H = gas.inviscid_flux(Q, gam)                              # [E][Np][j][5]
        if viscous:
            H = H - Fv
        Hhat = np.einsum('emdj,emjv->emdv', self.S, H)             # [E][Np][d][5]
        div = sum(np.einsum('mn,env->emv', self.Dop[d], Hhat[:, :, d, :]) for d in range(3))
        # Own normal flux at the flux points (interpolated transformed flux . outward normal).
        Fperp = np.stack([FACE_SIGN[f] * np.einsum('qm,emv->eqv', self.Lf[f], Hhat[:, :, FACE_AXIS[f], :])
                          for f in range(6)], axis=1)              # [E][6][Nf][5]
        # Common normal flux along side L's normal.
        FI = gas.common_flux(ph.inviscid_flux, QL, QR, self.nL, gam)
        if viscous:
            gL = gface[self.eL, self.fL]
            gR = gface[self.eR, self.fR][rows, self.perm]
            gc = np.where(up[:, None, None, None], gR, gL) if ldg else 0.5 * (gL + gR)
            nu_if = 0.5 * (nu_el[self.eL] + nu_el[self.eR])[:, None] * QI[..., 0]
            FI = FI - np.einsum('pqjv,pqj->pqv', gas.viscous_flux(QI, gc, gam, ph.R, ph.mu + nu_if, ph.Pr,
                                                                  kappa=kappa0 + nu_if * cp / PR_TURB), self.nL)
            if ldg:
                FI = FI + ph.ldg_tau * np.linalg.norm(self.nL, axis=-1)[..., None] * (QL - QR)
        Fc = np.empty_like(Fperp)
        Fc[self.eL, self.fL] = FI
        Fc[self.eR, self.fR] = -FI[rows, self.invperm]
        for k in range(len(self.bE)):
            e, f = self.bE[k], self.bF[k]
            n = self.nf[e, f]
            Qm = Qf[e, f]
            Fb = gas.common_flux(ph.inviscid_flux, Qm, ghosts[k], n, gam)
            if viscous:
                # Common gradient at a boundary: the interior side's face gradient.
                nb = nu_el[e] * bstates[k][..., 0]
                Fb = Fb - np.einsum('qjv,qj->qv', gas.viscous_flux(bstates[k], gface[e, f], gam, ph.R, ph.mu + nb, ph.Pr,
                                                                   kappa=kappa0 + nb * cp / PR_TURB), n)
                if ldg:
                    Fb = Fb + ph.ldg_tau * np.linalg.norm(n, axis=-1)[:, None] * (Qm - bstates[k])
            Fc[e, f] = Fb
        if magnitude:
            A = np.abs(Hhat)
            mag = sum(np.einsum('mn,env->emv', np.abs(self.Dop[d]), A[:, :, d, :]) for d in range(3))
            for f in range(6):
                own = np.einsum('qm,emv->eqv', np.abs(self.Lf[f]), A[:, :, FACE_AXIS[f], :])
                mag = mag + np.einsum('mq,eqv->emv', np.abs(self.Cf[f]), np.abs(Fc[:, f]) + own)
            return mag / self.detJ[..., None]
        corr = sum(self._lift(f, Fc[:, f] - Fperp[:, f]) for f in range(6))
        return -(div + corr) / self.detJ[..., None]

    # ------------------------------------------------------------------ time integration
    def rk44_step(self, Q, t, dt):
        """Classical four-stage Runge-Kutta step."""
        k1 = self.residual(Q, t)
        k2 = self.residual(Q + 0.5 * dt * k1, t + 0.5 * dt)
        k3 = self.residual(Q + 0.5 * dt * k2, t + 0.5 * dt)
        k4 = self.residual(Q + dt * k3, t + dt)
        return Q + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)

    def max_dt(self, Q, cfl):
        """dt = CFL min_e h_e / ((2p+1) max_pts(|u| + c)), h_e = vol_e^{1/3}."""
        rho, u, p = gas.primitives(Q, self.phys.gamma)
        lam = np.sqrt(np.sum(u * u, axis=-1)) + np.sqrt(self.phys.gamma * p / rho)
        return cfl * float(np.min(self.h / ((2 * self.p + 1) * np.max(lam, axis=1))))

    def integrate(self, Q, w=None):
        """Quadrature sum_e sum_m W_m |J|_m Q_m per variable (the discrete integral over the mesh)."""
        return np.einsum('m,em,emv->v', self.W, self.detJ, Q)
