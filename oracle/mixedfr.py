"""FR residual on mixed hexahedral / prismatic meshes (oracle; test infrastructure only).

The same semi-discretisation as `hexfr` (section "FR Algorithm", Eq. 1-3, BR2 viscous terms,
Rusanov flux, DG-equivalent correction) written with generic per-element-type operators:
  D_d       derivative along reference axis d at the solution points (Eq. 2 nodal basis),
  L_f       interpolation to the flux points of face f,
  C_f       divergence of face f's correction fields = DG lifting M^-1 E_f (exact mass matrix M,
            E_f[i][q] = integral over the reference face of phi_i times the face's nodal basis
            function q) -- the c = 0 (DG) choice, for hexahedra equal to the Radau construction;
            hexahedra also take a member c != 0 of the energy-stable family (phys.vcjh_c,
            basis.correction_right) through their 1D correction vectors, prisms only c = 0,
  N_f       outward reference normal of face f scaled by the reference face's measure per unit
            parameter area (the hypotenuse face of the prism: (1, 1, 0)).
Then grad_xi Q^C = D Q + sum_f C_f (Q^I - Q_f) N_f, F_perp = L_f (N_f . F^), the common flux uses
the area-scaled physical normal S^T N_f, and R = -|J|^-1 [sum_d D_d F^_d + sum_f C_f (F^I_perp -
F_perp)].

Prism: triangle (warp-and-blend nodes, module `tri`) x Gauss-Legendre line; 6-node linear map
with vertices (-1,-1,-1), (1,-1,-1), (-1,1,-1) and the same at zeta = +1 (VTK order).  Faces:
0 zeta=-1 and 1 zeta=+1 (triangles, flux points = the triangle nodes), 2 s=-1, 3 r+s=0, 4 r=-1
(quadrilaterals, flux points = Gauss-Legendre x Gauss-Legendre in (edge parameter, zeta)).
Interfaces are handled one by one (this module serves small meshes).
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from . import gas
from .basis import Basis1D
from .hexfr import HEX_REF_VERTS, boundary_states, trilinear_geometry
from .tri import Tri
from .curved import curved_geometry

PRISM_REF_VERTS = np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1], [1, -1, 1], [-1, 1, 1]], dtype=np.float64)


class ElemType:
    pass


def hex_type(p, curved=False, c=0.0):
    b = Basis1D(p, c)
    N = p + 1
    I = np.eye(N)
    t = ElemType()
    t.name, t.nv, t.Np = "hex", 8, N ** 3
    t.Dop = [np.kron(I, np.kron(I, b.D)), np.kron(I, np.kron(b.D, I)), np.kron(b.D, np.kron(I, I))]
    xi = b.nodes
    K, J, Ii = np.meshgrid(xi, xi, xi, indexing="ij")
    t.ref_sol = np.stack([Ii.ravel(), J.ravel(), K.ravel()], axis=1)
    t.W = np.kron(b.weights, np.kron(b.weights, b.weights))
    t.faces = []
    for f in range(6):
        d, s = f // 2, (1 if f % 2 else -1)
        row = (b.l_plus if s > 0 else b.l_minus)[None, :]
        col = (b.h_plus if s > 0 else b.h_minus)[:, None]
        if d == 0:
            L, C = np.kron(I, np.kron(I, row)), np.kron(I, np.kron(I, col))
        elif d == 1:
            L, C = np.kron(I, np.kron(row, I)), np.kron(I, np.kron(col, I))
        else:
            L, C = np.kron(row, np.kron(I, I)), np.kron(col, np.kron(I, I))
        tang = [a for a in range(3) if a != d]
        A, B = np.meshgrid(xi, xi, indexing="ij")
        pts = np.zeros((N * N, 3))
        pts[:, tang[0]], pts[:, tang[1]], pts[:, d] = B.ravel(), A.ravel(), s
        Nxi = np.zeros(3)
        Nxi[d] = s
        corners = np.where(HEX_REF_VERTS[:, d] == s)[0]
        t.faces.append(dict(L=L, C=C, N=Nxi, pts=pts, corners=corners, kind="quad"))
    t.geometry = lambda X, ref: trilinear_geometry(X, ref)
    if curved:
        t.nv, t.geometry = 27, curved_geometry("hex", p)
    return t


def prism_geometry(X, ref):
    """Physical points, |J| and S = |J| J^-1 of 6-node prisms at reference points ref [M][3]."""
    r, s, z = ref[:, 0], ref[:, 1], ref[:, 2]
    lam = np.stack([-(r + s) / 2, (1 + r) / 2, (1 + s) / 2], axis=1)          # [M][3]
    dlam = np.array([[-0.5, -0.5], [0.5, 0.0], [0.0, 0.5]])                  # d lam_v / d(r, s)
    lo, hi = (1 - z) / 2, (1 + z) / 2
    Nv = np.concatenate([lam * lo[:, None], lam * hi[:, None]], axis=1)      # [M][6]
    dN = np.zeros((len(r), 6, 3))
    for v in range(3):
        for a in range(2):
            dN[:, v, a] = dlam[v, a] * lo
            dN[:, v + 3, a] = dlam[v, a] * hi
        dN[:, v, 2] = -lam[:, v] / 2
        dN[:, v + 3, 2] = lam[:, v] / 2
    x = np.einsum('mv,evi->emi', Nv, X)
    J = np.einsum('mvb,evi->emib', dN, X)
    detJ = np.linalg.det(J)
    S = detJ[..., None, None] * np.linalg.inv(J)
    return x, detJ, S


def prism_type(p, curved=False):
    b = Basis1D(p)
    T = Tri(p)
    N, Nt = p + 1, T.Nt
    It, I = np.eye(Nt), np.eye(N)
    t = ElemType()
    t.name, t.nv, t.Np = "prism", 6, Nt * N
    t.Dop = [np.kron(I, T.Dr), np.kron(I, T.Ds), np.kron(b.D, It)]
    t.ref_sol = np.array([[T.rs[q, 0], T.rs[q, 1], b.nodes[k]] for k in range(N) for q in range(Nt)])
    wT = T.M @ np.ones(Nt)                                                   # int of each basis fn
    t.W = np.kron(b.weights, wT)
    Minv = np.linalg.inv(T.M)
    t.faces = []
    for s, row, col, corners in ((-1, b.l_minus, b.h_minus, [0, 1, 2]), (1, b.l_plus, b.h_plus, [3, 4, 5])):
        pts = np.array([[T.rs[q, 0], T.rs[q, 1], s] for q in range(Nt)], dtype=np.float64)
        t.faces.append(dict(L=np.kron(row[None, :], It), C=np.kron(col[:, None], It), N=np.array([0, 0, s], float),
                            pts=pts, corners=np.array(corners), kind="tri"))
    sig, w = b.nodes, b.weights
    edges = [(lambda x: np.stack([x, -np.ones_like(x)], 1), np.array([0.0, -1.0, 0.0]), [0, 1, 4, 3]),
             (lambda x: np.stack([-x, x], 1), np.array([1.0, 1.0, 0.0]), [1, 2, 5, 4]),
             (lambda x: np.stack([-np.ones_like(x), -x], 1), np.array([-1.0, 0.0, 0.0]), [2, 0, 3, 5])]
    for emap, Nxi, corners in edges:
        E = T.interp(emap(sig))                                              # [N][Nt]
        Ehat = E.T * w[None, :]                                              # int phi_t l_a dsigma
        rs = emap(sig)
        pts = np.array([[rs[a, 0], rs[a, 1], b.nodes[bb]] for bb in range(N) for a in range(N)])
        t.faces.append(dict(L=np.kron(I, E), C=np.kron(I, Minv @ Ehat), N=Nxi, pts=pts,
                            corners=np.array(corners), kind="quad"))
    t.geometry = prism_geometry
    if curved:
        t.nv, t.geometry = 18, curved_geometry("prism", p)
    return t


class MixedFR:
    """Oracle FR on a mesh of hexahedra (desc.hex) and prisms (desc.prism) at order p."""

    def __init__(self, desc, phys, p):
        self.phys, self.p = phys, p
        prism = getattr(desc, "prism", None)
        hexa = np.asarray(desc.hex, dtype=np.int64)
        pri = np.zeros((0, 6), np.int64) if prism is None else np.asarray(prism, dtype=np.int64)
        # 27-node hexahedra / 18-node prisms: quadratic maps with curl-form metrics.
        c = getattr(phys, "vcjh_c", 0.0)
        if c != 0.0 and len(pri) > 0:
            raise ValueError("the VCJH family with c != 0 is defined here for hexahedra only")
        self.types = [hex_type(p, curved=hexa.ndim == 2 and hexa.shape[1] == 27, c=c),
                      prism_type(p, curved=pri.ndim == 2 and pri.shape[1] == 18)]
        conn = [hexa.reshape(-1, self.types[0].nv), pri.reshape(-1, self.types[1].nv)]
        self.conn = conn
        self.x, self.detJ, self.S, self.nf, self.xf = [], [], [], [], []
        for t, cn in zip(self.types, conn):
            X = desc.xyz[cn]
            if len(cn) == 0:
                self.x.append(np.zeros((0, t.Np, 3)))
                self.detJ.append(np.zeros((0, t.Np)))
                self.S.append(np.zeros((0, t.Np, 3, 3)))
                self.nf.append([np.zeros((0, f["pts"].shape[0], 3)) for f in t.faces])
                self.xf.append([np.zeros((0, f["pts"].shape[0], 3)) for f in t.faces])
                continue
            x, dJ, S = t.geometry(X, t.ref_sol)
            if np.any(dJ <= 0):
                raise ValueError("non-positive Jacobian")
            self.x.append(x)
            self.detJ.append(dJ)
            self.S.append(S)
            nfs, xfs = [], []
            for f in t.faces:
                xf, _, Sf = t.geometry(X, f["pts"])
                xfs.append(xf)
                nfs.append(np.einsum('d,emdj->emj', f["N"], Sf))
            self.nf.append(nfs)
            self.xf.append(xfs)
        self._connect(desc)

    def _connect(self, desc):
        btag = {}
        for nodes, t in zip(desc.bface_nodes.tolist(), desc.bface_tag.tolist()):
            btag[tuple(sorted(v for v in nodes if v >= 0))] = int(t)
        shift_of = {}
        for per in desc.periodic:
            shift_of[per.tag_b] = np.asarray(per.t, dtype=np.float64)
            shift_of.setdefault(per.tag_a, np.zeros(3))
        bc_of = {bc.tag: bc for bc in desc.bcs}
        keys, recs, bfaces = [], [], []
        for ti, (t, cn) in enumerate(zip(self.types, self.conn)):
            for e in range(len(cn)):
                for fi, f in enumerate(t.faces):
                    nodes = cn[e, f["corners"]]
                    tag = btag.get(tuple(sorted(nodes.tolist())), 0)
                    cent = desc.xyz[nodes].mean(axis=0)
                    if tag and tag not in shift_of:
                        if tag not in bc_of:
                            raise ValueError("boundary tag without condition")
                        bfaces.append((ti, e, fi, bc_of[tag]))
                        continue
                    keys.append(cent - (shift_of[tag] if tag else 0.0))
                    recs.append((ti, e, fi, shift_of[tag] if tag else np.zeros(3)))
        hmin = min(float(np.min(np.abs(dJ)) ** (1 / 3)) for dJ in self.detJ if len(dJ))
        pairs = sorted(cKDTree(np.array(keys)).query_pairs(r=1e-6 * hmin))
        if 2 * len(pairs) != len(recs):
            raise ValueError("unmatched faces")
        self.ifaces = []
        for a, bb in pairs:
            (tL, eL, fL, sL), (tR, eR, fR, sR) = recs[a], recs[bb]
            xL = self.xf[tL][fL][eL] - sL
            xR = self.xf[tR][fR][eR] - sR
            dist = np.linalg.norm(xL[:, None, :] - xR[None, :, :], axis=-1)
            perm = np.argmin(dist, axis=1)
            if dist[np.arange(len(perm)), perm].max() > 1e-6 * hmin:
                raise ValueError("flux points do not match")
            self.ifaces.append((tL, eL, fL, tR, eR, fR, perm))
        self.bfaces = bfaces
        self.h = [np.cbrt(np.einsum('m,em->e', t.W, dJ)) for t, dJ in zip(self.types, self.detJ)]

    def set_source(self, accel=None, sigma=None, Q_ref=None):
        """Source term S of Eq. 3 added to the residual: body acceleration g (S = (0, rho g,
        rho u . g)) and a sponge S = -sigma(x) (Q - Q_ref(x)); sigma and Q_ref are lists per element
        type ([E][Np] and [E][Np][5]).  None switches a part off."""
        self.accel = None if accel is None else np.asarray(accel, dtype=np.float64)
        self.sigma = sigma
        self.Q_ref = Q_ref

    def _source(self, ti, Q):
        S = np.zeros_like(Q)
        if getattr(self, "accel", None) is not None:
            S[..., 1:4] = Q[..., 0:1] * self.accel
            S[..., 4] = Q[..., 1:4] @ self.accel
        if getattr(self, "sigma", None) is not None:
            S -= self.sigma[ti][..., None] * (Q - self.Q_ref[ti])
        return S

    def solution_points(self):
        return [x.copy() for x in self.x]

    def residual(self, Qs, magnitude=False):
        """Qs: [Q_hex [E_h][Np_h][5], Q_prism [E_p][Np_p][5]] -> residuals in the same layout.

        With magnitude=True it returns instead the entrywise magnitude of the final sum,
        |J|^-1 [sum_d |D_d| |F^_d| + sum_f |C_f| (|F^I_perp| + |L_f| sum_d |N_f,d| |F^_d|)], the scale
        of the rounding error of any evaluation order (used for tolerances).
        """
        ph = self.phys
        gam = ph.gamma
        visc = ph.viscous != 0 and ph.mu != 0.0
        ldg = visc and ph.viscous == 2
        T = self.types
        Qf = [[np.einsum('qm,emv->eqv', f["L"], Q) for f in t.faces] for t, Q in zip(T, Qs)]
        dQ = [[np.zeros_like(a) for a in qf] for qf in Qf]
        Qc_if, gh, ups = [], [], []
        for (tL, eL, fL, tR, eR, fR, perm) in self.ifaces:
            qL, qR = Qf[tL][fL][eL], Qf[tR][fR][eR][perm]
            # LDG: the side whose face normal points along gas.LDG_SWITCH supplies Q^I.
            up = bool(self.nf[tL][fL][eL].sum(axis=0) @ gas.LDG_SWITCH > 0)
            ups.append(up)
            qI = (qL if up else qR) if ldg else 0.5 * (qL + qR)
            dQ[tL][fL][eL] = qI - qL
            dQ[tR][fR][eR][perm] = qI - qR
            Qc_if.append(qI)
        ghosts, bst = [], []
        for (ti, e, fi, bc) in self.bfaces:
            gh, qi = boundary_states(bc.kind, np.asarray(bc.params, dtype=np.float64), Qf[ti][fi][e],
                                     self.nf[ti][fi][e], ph.gamma, ph.R)
            dQ[ti][fi][e] = qi - Qf[ti][fi][e]
            ghosts.append(gh)
            bst.append(qi)
        grads, gfaces, Hhat = [], [], []
        for ti, (t, Q) in enumerate(zip(T, Qs)):
            Sinv = self.S[ti] / self.detJ[ti][..., None, None]
            gu = np.stack([np.einsum('mn,env->emv', t.Dop[d], Q) for d in range(3)], axis=2)
            gc = gu.copy()
            lifts = []
            for fi, f in enumerate(t.faces):
                lf = np.einsum('mq,eqv->emv', f["C"], dQ[ti][fi])
                lifts.append(lf)
                gc += lf[:, :, None, :] * f["N"][None, None, :, None]
            grad = np.einsum('emdj,emdv->emjv', Sinv, gc)
            gunc = np.einsum('emdj,emdv->emjv', Sinv, gu)
            gf = []
            for fi, f in enumerate(t.faces):
                if ldg:
                    gf.append(np.einsum('qm,emjv->eqjv', f["L"], grad))
                    continue
                rf = np.einsum('emdj,d,emv->emjv', Sinv, f["N"], lifts[fi])
                gf.append(np.einsum('qm,emjv->eqjv', f["L"], gunc + ph.br2_eta * rf))
            H = gas.inviscid_flux(Q, gam)
            if visc:
                H = H - gas.viscous_flux(Q, grad, gam, ph.R, ph.mu, ph.Pr)
            grads.append(grad)
            gfaces.append(gf)
            Hhat.append(np.einsum('emdj,emjv->emdv', self.S[ti], H))
        Fc = [[np.zeros_like(a) for a in qf] for qf in Qf]
        for k, (tL, eL, fL, tR, eR, fR, perm) in enumerate(self.ifaces):
            qL, qR = Qf[tL][fL][eL], Qf[tR][fR][eR][perm]
            n = self.nf[tL][fL][eL]
            F = gas.common_flux(ph.inviscid_flux, qL, qR, n, gam)
            if visc:
                gl, gr = gfaces[tL][fL][eL], gfaces[tR][fR][eR][perm]
                g = (gr if ups[k] else gl) if ldg else 0.5 * (gl + gr)
                F = F - np.einsum('qjv,qj->qv', gas.viscous_flux(Qc_if[k], g, gam, ph.R, ph.mu, ph.Pr), n)
                if ldg:
                    F = F + ph.ldg_tau * np.linalg.norm(n, axis=-1)[:, None] * (qL - qR)
            Fc[tL][fL][eL] = F
            Fc[tR][fR][eR][perm] = -F
        for k, (ti, e, fi, bc) in enumerate(self.bfaces):
            n = self.nf[ti][fi][e]
            F = gas.common_flux(ph.inviscid_flux, Qf[ti][fi][e], ghosts[k], n, gam)
            if visc:
                F = F - np.einsum('qjv,qj->qv', gas.viscous_flux(bst[k], gfaces[ti][fi][e], gam, ph.R, ph.mu, ph.Pr), n)
                if ldg:
                    F = F + ph.ldg_tau * np.linalg.norm(n, axis=-1)[:, None] * (Qf[ti][fi][e] - bst[k])
            Fc[ti][fi][e] = F
        out = []
        if magnitude:
            for ti, t in enumerate(T):
                A = np.abs(Hhat[ti])
                mag = sum(np.einsum('mn,env->emv', np.abs(t.Dop[d]), A[:, :, d, :]) for d in range(3))
                for fi, f in enumerate(t.faces):
                    own = np.einsum('qm,emv->eqv', np.abs(f["L"]), np.einsum('d,emdv->emv', np.abs(f["N"]), A))
                    mag = mag + np.einsum('mq,eqv->emv', np.abs(f["C"]), np.abs(Fc[ti][fi]) + own)
                out.append(mag / self.detJ[ti][..., None] + np.abs(self._source(ti, Qs[ti])))
            return out
        for ti, t in enumerate(T):
            R = sum(np.einsum('mn,env->emv', t.Dop[d], Hhat[ti][:, :, d, :]) for d in range(3))
            for fi, f in enumerate(t.faces):
                own = np.einsum('qm,emv->eqv', f["L"], np.einsum('d,emdv->emv', f["N"], Hhat[ti]))
                R = R + np.einsum('mq,eqv->emv', f["C"], Fc[ti][fi] - own)
            out.append(-R / self.detJ[ti][..., None] + self._source(ti, Qs[ti]))
        return out

    def integrate(self, Rs):
        return sum(np.einsum('m,em,emv->v', t.W, dJ, R) for t, dJ, R in zip(self.types, self.detJ, Rs))
