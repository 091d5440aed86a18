"""Pins of the mixed hexahedral/prismatic oracle (CPU only)."""
import numpy as np
import pytest

from paper_2308_06605_gb300 import inputs as I
from oracle import gas
from oracle.hexfr import HexFR
from oracle.mixedfr import MixedFR, prism_type
from oracle.tri import Tri

G = 1.4


def test_equals_hex_oracle_on_hex_meshes():
    d = I.hex_box_mesh((3, 3, 3), seed=2, rotate=True, shuffle=True, perturb=0.1)
    ph = I.tgv_physics(Ma=0.2, Re=300.0)
    mh, mm = HexFR(d, ph, 3), MixedFR(d, ph, 3)
    Q = I.tgv_state(mh.x, Ma=0.2, perturb=1e-2)
    R1 = mh.residual(Q)
    R2 = mm.residual([Q, np.zeros((0, mm.types[1].Np, 5))])[0]
    np.testing.assert_allclose(R2, R1, rtol=0, atol=1e-13 * np.abs(R1).max())
    # The magnitude scale reduces to the hexahedral oracle's on hexahedral meshes.
    S1 = mh.residual(Q, magnitude=True)
    S2 = mm.residual([Q, np.zeros((0, mm.types[1].Np, 5))], magnitude=True)[0]
    np.testing.assert_allclose(S2, S1, rtol=1e-13)


def test_magnitude_bounds_the_residual():
    d = I.hex_box_mesh((3, 3, 2), prisms="checker", seed=3, rotate=True, perturb=0.05)
    ph = I.tgv_physics(Ma=0.2, Re=300.0)
    m = MixedFR(d, ph, 3)
    Qs = [I.tgv_state(x, Ma=0.2, perturb=1e-2) for x in m.x]
    for R, S in zip(m.residual(Qs), m.residual(Qs, magnitude=True)):
        assert np.all(np.abs(R) <= S * (1 + 1e-12))
        assert np.all(S > 0)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_prism_lifting_is_dg_lifting(p):
    """C_f = M^-1 E_f with E_f from an independent over-integrated face quadrature of the nodal
    basis (collapsed-coordinate rule for the triangle, Gauss rule on the faces)."""
    t = prism_type(p)
    T = Tri(p)
    N, Nt = p + 1, T.Nt
    xq, wq = np.polynomial.legendre.leggauss(N + 3)
    # 3D mass matrix by over-integration on the prism (collapsed triangle x Gauss line)
    U, S = np.meshgrid(xq, xq, indexing="ij")
    R = (1 + U) * (1 - S) / 2 - 1
    Wt = (np.outer(wq, wq) * (1 - S) / 2).ravel()
    Lt = T.interp(np.stack([R.ravel(), S.ravel()], 1))                      # [Q][Nt]
    xn, _ = np.polynomial.legendre.leggauss(N)
    lz = np.array([[np.prod([(z - xn[m]) / (xn[k] - xn[m]) for m in range(N) if m != k]) for k in range(N)] for z in xq])
    phi = np.einsum('qt,zk->qzkt', Lt, lz).reshape(len(Wt) * len(xq), N * Nt)    # basis index k*Nt + t
    wts = np.einsum('q,z->qz', Wt, wq).ravel()
    M = phi.T @ (wts[:, None] * phi)
    for f in t.faces[2:]:                                                     # quad faces
        # face nodal basis (Gauss points in sigma and zeta) at a finer face rule
        Ne = t.faces[2]["pts"].shape[0]
        sig = xq
        E = np.zeros((N * Nt, Ne))
        # reconstruct the face map from its flux points: (r, s) linear in sigma
        pts = f["pts"].reshape(N, N, 3)[0, :, :2]                             # zeta-index 0, sigma varies
        a0, a1 = pts[0], pts[-1]
        x0, x1 = xn[0], xn[-1]
        for ia, sg in enumerate(sig):
            rs = a0 + (a1 - a0) * (sg - x0) / (x1 - x0)
            la = np.array([np.prod([(sg - xn[m]) / (xn[k] - xn[m]) for m in range(N) if m != k]) for k in range(N)])
            phit = T.interp(rs[None, :])[0]
            for iz, z in enumerate(xq):
                lzz = lz[iz]
                E += wq[ia] * wq[iz] * np.outer(np.kron(lzz, phit), np.kron(lzz, la))
        np.testing.assert_allclose(f["C"], np.linalg.solve(M, E), atol=1e-11)


@pytest.mark.parametrize("prisms", ["all", "checker"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_free_stream_and_conservation(prisms, p):
    ph = I.tgv_physics(Ma=0.2, Re=300.0)
    d = I.hex_box_mesh((3, 3, 2), seed=p, rotate=True, shuffle=True, prisms=prisms, perturb=0.1 if p > 1 else 0.0)
    m = MixedFR(d, ph, p)
    R = m.residual([I.uniform_state(x.shape[:2]) for x in m.x])
    assert max(np.abs(r).max() for r in R if r.size) <= 1e-13 * 1.5 / min(h.min() for h in m.h if len(h))
    R = m.residual([I.tgv_state(x, Ma=0.2, perturb=1e-2, seed=p) for x in m.x])
    s = np.abs(m.integrate(R))
    a = sum(np.einsum('m,em,emv->v', t.W, dJ, np.abs(r)) for t, dJ, r in zip(m.types, m.detJ, R))
    assert np.all(s <= 1e-12 * a)


def test_orientation_invariance_mixed():
    ph = I.tgv_physics(Ma=0.2, Re=300.0)
    ma = MixedFR(I.hex_box_mesh((3, 3, 2), prisms="checker"), ph, 2)
    mb = MixedFR(I.hex_box_mesh((3, 3, 2), prisms="checker", seed=5, rotate=True, shuffle=True), ph, 2)
    Ra = ma.residual([I.tgv_state(x, Ma=0.2, perturb=1e-2) for x in ma.x])
    Rb = mb.residual([I.tgv_state(x, Ma=0.2, perturb=1e-2) for x in mb.x])
    # Triangle nodes include edge points shared by neighbouring prisms: match elements by
    # centroid first, then points within the element.
    from scipy.spatial import cKDTree
    for t in range(2):
        if ma.x[t].size == 0:
            continue
        ei = cKDTree(mb.x[t].mean(axis=1)).query(ma.x[t].mean(axis=1))[1]
        for e in range(ma.x[t].shape[0]):
            d, i = cKDTree(mb.x[t][ei[e]]).query(ma.x[t][e])
            assert d.max() < 1e-9
            np.testing.assert_allclose(Rb[t][ei[e]][i], Ra[t][e], rtol=0, atol=1e-12 * np.abs(Ra[t]).max())


@pytest.mark.parametrize("prisms", ["all", "checker"])
def test_polynomial_exactness_with_dirichlet(prisms):
    """rho = 1, u = a + b x, p = P0: fluxes of degree <= 3, so R = -div(F - F_v) exactly (p = 3);
    the prisms' hypotenuse faces see the x-flux through their diagonal normals."""
    a, b, P0, mu = 0.3, 0.2, 2.0, 0.05
    lo, hi = (0.0, 0.0, 0.0), (1.5, 1.0, 1.0)
    state = lambda X: I.conserved(np.ones_like(X), a + b * X, 0 * X, 0 * X, P0 * np.ones_like(X), G)  # noqa: E731
    d = I.hex_box_mesh((3, 2, 2), lo=lo, hi=hi, periodic=(False, True, True), prisms=prisms, seed=1, rotate=True,
                       wall_tags={1: (I.BC_DIRICHLET, tuple(state(np.array(lo[0])))),
                                  2: (I.BC_DIRICHLET, tuple(state(np.array(hi[0]))))})
    m = MixedFR(d, I.Physics(gamma=G, R=1.0, mu=mu, Pr=0.71, viscous=1), 3)
    R = m.residual([state(x[..., 0]) for x in m.x])
    for x, r in zip(m.x, R):
        u = a + b * x[..., 0]
        want = np.zeros(r.shape)
        want[..., 0] = -b
        want[..., 1] = -2 * b * u
        want[..., 4] = -(G * P0 * b / (G - 1) + 1.5 * b * u * u) + 4.0 / 3.0 * mu * b * b
        np.testing.assert_allclose(r, want, rtol=0, atol=1e-11 * 2.0)


@pytest.mark.parametrize("kinds", [
    ((I.BC_WALL_ISOTHERMAL, (1.1,)), (I.BC_CHAR_OUTFLOW, (0.7,))),
    ((I.BC_CHAR_INFLOW, (0.9, 1.05, 1.0, 0.2, 0.0)), (I.BC_WALL_ISOTHERMAL, (0.9,)))])
def test_boundary_conditions_equal_hex_oracle(kinds):
    """Walls and characteristic boundaries: on hexahedral meshes the mixed-element oracle equals the
    hexahedral one (whose boundary states are pinned separately)."""
    d = I.hex_box_mesh((3, 2, 2), hi=(2.0, 1.0, 1.0), periodic=(False, True, True),
                       wall_tags={1: kinds[0], 2: kinds[1]}, seed=3, rotate=True, perturb=0.1)
    ph = I.Physics(gamma=1.4, R=1.0, mu=0.02, Pr=0.71, viscous=1)
    mh, mm = HexFR(d, ph, 3), MixedFR(d, ph, 3)
    Q = I.conserved(1 + 0.1 * np.sin(mh.x[..., 0]), 0.2 + 0 * mh.x[..., 0], 0.1 + 0 * mh.x[..., 0],
                    0.05 * np.sin(2 * np.pi * mh.x[..., 2]), 0.7 + 0.02 * mh.x[..., 0], 1.4)
    R1 = mh.residual(Q)
    R2 = mm.residual([Q, np.zeros((0, mm.types[1].Np, 5))])[0]
    np.testing.assert_allclose(R2, R1, rtol=0, atol=1e-13 * np.abs(R1).max())


def test_walls_on_triangular_faces_keep_quiescent_gas_at_rest():
    """Gas at rest at the wall temperature between isothermal walls through triangular faces:
    an exact steady state (zero residual)."""
    T_w = 1.2
    d = I.hex_box_mesh((2, 2, 3), hi=(1.0, 1.0, 1.5), periodic=(True, True, False), prisms="checker", seed=2,
                       rotate=True, perturb=0.1,
                       wall_tags={5: (I.BC_WALL_ISOTHERMAL, (T_w,)), 6: (I.BC_WALL_ISOTHERMAL, (T_w,))})
    ph = I.Physics(gamma=1.4, R=1.0, mu=0.05, Pr=0.71, viscous=1)
    m = MixedFR(d, ph, 3)
    Qs = [I.conserved(np.ones(x.shape[:2]), 0 * x[..., 0], 0 * x[..., 0], 0 * x[..., 0], T_w * np.ones(x.shape[:2]), 1.4)
          for x in m.x]
    for R in m.residual(Qs):
        assert np.abs(R).max() <= 1e-12
