"""Brute-force pin of the oracle's hexahedral Navier-Stokes residual on 1- and 2-element meshes.

An independent restatement at 40 significant digits (mpmath): nodal DG in WEAK form with the
exact (non-lumped) mass matrix and over-integrated quadrature, on sheared affine periodic
lattices.  With the c = 0 correction the FR scheme of arXiv 2308.06605 (section "FR Algorithm",
Eq. 3) equals this strong/weak-form DG with collocated fluxes:
    M dQ/dt = int grad(phi) . H^delta dx - sum_faces int phi (H^I . n)^delta dS,
with the BR2 gradient  M G = int phi grad Q^delta + sum_f int phi dQ^delta n dS  and the face
lifting  M r_f = int_f phi dQ^delta n dS.  Nothing here calls the oracle's basis, operators,
connectivity or gas functions; only the resulting residual is compared.
"""
import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp

from paper_2308_06605_gb300 import inputs as I  # noqa: E402
from oracle.hexfr import HexFR  # noqa: E402
from oracle.weakdg_mp import brute_force_residual  # noqa: E402


SHEAR = [[1.0, 0.21, -0.13], [0.07, 0.93, 0.18], [-0.11, 0.05, 1.08]]


@pytest.mark.parametrize("p,n1,viscous", [(1, 1, True), (1, 2, True), (2, 1, True), (2, 2, False)])
def test_oracle_matches_mpmath_weak_form(p, n1, viscous):
    hbox = (0.9 * n1, 1.1, 0.8)
    desc = I.hex_box_mesh((n1, 1, 1), lo=(0.0, 0.0, 0.0), hi=hbox, affine=SHEAR)
    phys = I.Physics(gamma=1.4, R=1.0, mu=0.05 if viscous else 0.0, Pr=0.71, viscous=1 if viscous else 0, br2_eta=6.0)
    ora = HexFR(desc, phys, p)
    rng = np.random.default_rng(10 * p + n1)
    Np = (p + 1) ** 3
    rho = 1.0 + 0.2 * rng.uniform(-1, 1, (n1, Np))
    vel = 0.4 * rng.uniform(-1, 1, (n1, Np, 3))
    pr = 1.0 + 0.2 * rng.uniform(-1, 1, (n1, Np))
    Q = I.conserved(rho, vel[..., 0], vel[..., 1], vel[..., 2], pr, 1.4)
    R_ora = ora.residual(Q)
    hcell = (hbox[0] / n1, hbox[1], hbox[2])
    R_bf = brute_force_residual(Q, p, n1, SHEAR, hcell, phys.gamma, 1, phys.mu, phys.Pr, 6, viscous)
    scale = np.abs(R_bf).max(axis=(0, 1))
    err = np.abs(R_ora - R_bf).max(axis=(0, 1)) / scale
    assert np.all(err < 1e-13), err
