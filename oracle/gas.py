"""Ideal-gas compressible Navier-Stokes fluxes (oracle; test infrastructure only).

Conserved variables Q = (rho, rho u, rho v, rho w, E) on the last axis.  Physical fluxes are
returned as [..., 3, 5] arrays: entry [..., j, v] is the flux of variable v in direction x_j.
Eq. 1 of arXiv 2308.06605 writes the system as dQ/dt + div(F + G) = S with F the inviscid and G
the viscous flux; here G = -F_v with F_v the usual viscous flux (Stokes hypothesis, constant
viscosity mu, Fourier heat flux with conductivity kappa = mu gamma R / ((gamma - 1) Pr)).
"""
from __future__ import annotations

import numpy as np


def primitives(Q, gamma):
    rho = Q[..., 0]
    u = Q[..., 1:4] / rho[..., None]
    p = (gamma - 1.0) * (Q[..., 4] - 0.5 * rho * np.sum(u * u, axis=-1))
    return rho, u, p


def inviscid_flux(Q, gamma):
    """F[..., j, :] = (rho u_j, rho u u_j + p e_j, (E + p) u_j)."""
    rho, u, p = primitives(Q, gamma)
    E = Q[..., 4]
    F = np.empty(Q.shape[:-1] + (3, 5))
    for j in range(3):
        F[..., j, 0] = rho * u[..., j]
        for i in range(3):
            F[..., j, 1 + i] = rho * u[..., i] * u[..., j] + (p if i == j else 0.0)
        F[..., j, 4] = (E + p) * u[..., j]
    return F


def viscous_flux(Q, gradQ, gamma, R, mu, Pr, kappa=None):
    """F_v[..., j, :] = (0, tau_xj, tau_yj, tau_zj, u_i tau_ij + kappa dT/dx_j).

    gradQ[..., j, v] = dQ_v/dx_j.  Velocity and temperature gradients follow from the chain
    rule: du_i/dx_j = (d(rho u_i)/dx_j - u_i drho/dx_j)/rho and, with T = (gamma-1)/R (E/rho -
    |u|^2/2), dT/dx_j = (gamma-1)/R [ (dE/dx_j - (E/rho) drho/dx_j)/rho - u_i du_i/dx_j ].
    mu (and kappa, default mu cp / Pr) may be arrays broadcasting against Q[..., 0].
    """
    rho, u, _ = primitives(Q, gamma)
    E = Q[..., 4]
    if kappa is None:
        kappa = mu * gamma * R / ((gamma - 1.0) * Pr)
    gu = np.empty(Q.shape[:-1] + (3, 3))           # gu[..., i, j] = du_i/dx_j
    for i in range(3):
        for j in range(3):
            gu[..., i, j] = (gradQ[..., j, 1 + i] - u[..., i] * gradQ[..., j, 0]) / rho
    gT = np.empty(Q.shape[:-1] + (3,))
    for j in range(3):
        gT[..., j] = (gamma - 1.0) / R * ((gradQ[..., j, 4] - E / rho * gradQ[..., j, 0]) / rho
                                          - np.sum(u * gu[..., :, j], axis=-1))
    divu = gu[..., 0, 0] + gu[..., 1, 1] + gu[..., 2, 2]
    tau = np.empty(Q.shape[:-1] + (3, 3))
    for i in range(3):
        for j in range(3):
            tau[..., i, j] = mu * (gu[..., i, j] + gu[..., j, i] - (2.0 / 3.0 if i == j else 0.0) * divu)
    Fv = np.zeros(Q.shape[:-1] + (3, 5))
    for j in range(3):
        for i in range(3):
            Fv[..., j, 1 + i] = tau[..., i, j]
        Fv[..., j, 4] = np.sum(u * tau[..., :, j], axis=-1) + kappa * gT[..., j]
    return Fv


def sound_speed(Q, gamma):
    rho, _, p = primitives(Q, gamma)
    return np.sqrt(gamma * p / rho)


def rusanov(QL, QR, n, gamma):
    """Rusanov (local Lax-Friedrichs) common flux dotted with the (area-scaled) normal n of side L:
    1/2 (F(QL) + F(QR)) . n - 1/2 lambda |n| (QR - QL), lambda = max over sides of |u.n^| + c."""
    FL = np.einsum('...jv,...j->...v', inviscid_flux(QL, gamma), n)
    FR = np.einsum('...jv,...j->...v', inviscid_flux(QR, gamma), n)
    nmag = np.sqrt(np.sum(n * n, axis=-1))
    nh = n / nmag[..., None]
    _, uL, _ = primitives(QL, gamma)
    _, uR, _ = primitives(QR, gamma)
    lam = np.maximum(np.abs(np.sum(uL * nh, axis=-1)) + sound_speed(QL, gamma),
                     np.abs(np.sum(uR * nh, axis=-1)) + sound_speed(QR, gamma))
    return 0.5 * (FL + FR) - 0.5 * (lam * nmag)[..., None] * (QR - QL)


def roe(QL, QR, n, gamma, delta=0.1):
    """Roe's approximate Riemann flux (Roe 1981) dotted with the area-scaled normal n of side L:
    1/2 (F(QL) + F(QR)) . n - 1/2 |n| sum_k |lambda_k| alpha_k r_k over the waves of the Jacobian at
    the Roe average (density-weighted velocity and total enthalpy), with Harten's entropy fix
    |lambda| -> (lambda^2 + d^2) / (2 d) for |lambda| < d, d = delta * c~ on the acoustic waves.
    Waves: acoustic u.n^ -/+ c with strengths (dp -/+ rho c du_n) / (2 c^2), entropy u.n^ with
    drho - dp / c^2, shear u.n^ carrying rho (du - du_n n^)."""
    FL = np.einsum('...jv,...j->...v', inviscid_flux(QL, gamma), n)
    FR = np.einsum('...jv,...j->...v', inviscid_flux(QR, gamma), n)
    return 0.5 * (FL + FR) - 0.5 * roe_dissipation(QL, QR, n, gamma, delta, absolute=True)


def roe_dissipation(QL, QR, n, gamma, delta=0.1, absolute=True):
    """|n| sum_k f(lambda_k) alpha_k r_k with f = |.| (entropy-fixed) or, absolute=False, the
    identity (then the sum is A(Q~) (QR - QL) |n|, which for the Roe average equals
    (F(QR) - F(QL)) . n: Roe's property U, used as a pin)."""
    nmag = np.sqrt(np.sum(n * n, axis=-1))
    nh = n / nmag[..., None]
    rL, uL, pL = primitives(QL, gamma)
    rR, uR, pR = primitives(QR, gamma)
    HL = (QL[..., 4] + pL) / rL
    HR = (QR[..., 4] + pR) / rR
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    r = sL * sR
    u = (sL[..., None] * uL + sR[..., None] * uR) / (sL + sR)[..., None]
    H = (sL * HL + sR * HR) / (sL + sR)
    q2 = np.sum(u * u, axis=-1)
    c = np.sqrt((gamma - 1.0) * (H - 0.5 * q2))
    un = np.sum(u * nh, axis=-1)
    dr = rR - rL
    dp = pR - pL
    du = uR - uL
    dun = np.sum(du * nh, axis=-1)
    a1 = (dp - r * c * dun) / (2.0 * c * c)
    a2 = dr - dp / (c * c)
    a3 = (dp + r * c * dun) / (2.0 * c * c)
    lam1, lam2, lam3 = un - c, un, un + c
    if absolute:
        def fix(lam):
            d = delta * c
            a = np.abs(lam)
            return np.where(a < d, (lam * lam + d * d) / (2.0 * d), a)
        l1, l2, l3 = fix(lam1), np.abs(lam2), fix(lam3)
    else:
        l1, l2, l3 = lam1, lam2, lam3
    out = np.zeros(QL.shape)
    # acoustic waves
    for lam, a, s in ((l1, a1, -1.0), (l3, a3, 1.0)):
        out[..., 0] += lam * a
        out[..., 1:4] += (lam * a)[..., None] * (u + s * c[..., None] * nh)
        out[..., 4] += lam * a * (H + s * c * un)
    # entropy and shear waves (both travel at u.n^)
    shear = r[..., None] * (du - dun[..., None] * nh)
    out[..., 0] += l2 * a2
    out[..., 1:4] += l2[..., None] * (a2[..., None] * u + shear)
    out[..., 4] += l2 * (a2 * 0.5 * q2 + np.sum(u * shear, axis=-1))
    return nmag[..., None] * out


def common_flux(kind, QL, QR, n, gamma):
    """Inviscid common flux: kind 0 = Rusanov, 1 = Roe."""
    return roe(QL, QR, n, gamma) if kind == 1 else rusanov(QL, QR, n, gamma)


# LDG (Cockburn & Shu; the paper's viscous scheme via Huynh 2009): at each interface one side
# supplies the common solution and the other the common gradient.  The choice is geometric: the
# side whose outward normal, summed over the face, points along LDG_SWITCH supplies Q^I.
LDG_SWITCH = np.array([1.0, np.sqrt(2.0) / 2.0, np.sqrt(3.0) / 4.0])
