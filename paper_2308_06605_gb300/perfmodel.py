"""Algorithmic work per solution point of one residual evaluation + RK stage (hexahedra).

FLOP accounting follows the paper's convention (section "FLOPs Measurement"): contractions
count 2 per multiply-add of the operator actually applied (sum-factorised 1D operators here),
pointwise kernels count the operations of the algorithm.  Bytes are the algorithmic DRAM traffic
of each kernel of the FP64 pipeline (every array read or written once per launch, no re-reads).
Per-point figures for a periodic hexahedral mesh: 6 N^2 face points and 3 N^2 interface points
per element of N^3 solution points.
"""
from __future__ import annotations

KERNELS = ("interp_faces", "volume", "iface_flux", "correct")

# Pointwise operation counts (FP64 adds, multiplies, FMAs as 2, divisions/square roots as 1)
# read off the kernels' arithmetic.
_INVISCID = 22          # velocities (3 + 1 reciprocal), pressure (7), three flux vectors (11)
_VISCOUS = 98           # velocity/temperature gradients (39), stress (27), energy flux (24), misc
_TRANSFORM = 90         # F^_d = sum_j S_dj H_j: 15 x 3 FMAs
_PHYS_GRAD = 189        # two J^-T products (2 x 15 x 3 FMAs) + 9 metric scalings
_RUSANOV = 70           # two normal fluxes (2 x 26), |n|, wave speeds, dissipation (15)
_VISC_COMMON = 163      # averages (20 x 2), viscous flux (98), normal projection (15 x 2)


def flops_per_point(p: int, viscous: bool = True) -> dict:
    N = p + 1
    fp_pt = 6.0 / N          # face points per solution point
    if_pt = 3.0 / N          # interface points per solution point
    f = {}
    f["interp_faces"] = fp_pt * 5 * 2 * N
    vol = 2 * 3 * 5 * N                       # divergence, sum-factorised (Dt along 3 axes)
    vol += _INVISCID + _TRANSFORM
    if viscous:
        vol += 2 * 3 * 5 * N                  # reference gradient
        vol += 3 * 5 * 2 * 2                  # gradient correction from the two faces per axis
        vol += fp_pt * 5 * 2                  # jumps at the flux points
        vol += _PHYS_GRAD + _VISCOUS
        vol += fp_pt * 15 * (2 * N + 2)       # gradient traces: interpolation + eta * lift
    f["volume"] = vol
    f["iface_flux"] = if_pt * (_RUSANOV + (_VISC_COMMON if viscous else 0))
    f["correct"] = 6 * 5 * 2 + 5 + 5 * 4      # common-flux correction, scaling, RK stage update
    return f


def volume_split(p: int) -> tuple:
    """(flops of the viscous branch, flops of the rest) per point of the volume kernel: the branch
    FR_PREC_MIXED_VF32 runs in FP32 (reference gradient, its correction, the jumps, the physical
    gradient, the stress and heat flux, the gradient traces) and the rest (inviscid fluxes,
    transformation, divergence) in double-float."""
    N = p + 1
    fp_pt = 6.0 / N
    visc = 2 * 3 * 5 * N + 3 * 5 * 2 * 2 + fp_pt * 5 * 2 + _PHYS_GRAD + _VISCOUS + fp_pt * 15 * (2 * N + 2)
    rest = 2 * 3 * 5 * N + _INVISCID + _TRANSFORM
    return visc, rest


def mixed_alu_peak(p: int, df_peak: float, fp32_peak: float, fp32_viscous: bool) -> float:
    """Algorithmic-flop peak of the mixed volume kernel for its arithmetic mix: all double-float
    (df_peak), or the viscous branch at the FP32 rate and the rest in double-float (the time of
    each part at its own peak, added)."""
    if not fp32_viscous:
        return df_peak
    visc, rest = volume_split(p)
    return (visc + rest) / (rest / df_peak + visc / fp32_peak)


def bytes_per_point(p: int, viscous: bool = True, mode: str = "rk") -> dict:
    N = p + 1
    Np, Nf = N ** 3, N ** 2
    per_el = lambda doubles: 8.0 * doubles / Np          # noqa: E731  element-level arrays
    b = {}
    b["interp_faces"] = per_el(5 * Np) + per_el(6 * Nf * 5)
    vol = per_el(5 * Np) + per_el(10 * Np) + per_el(5 * Np)          # Q, metrics, Rpart
    if viscous:
        vol += per_el(2 * 6 * Nf * 5)                                 # own + other traces
        vol += per_el(6 * 3 * Nf) + per_el(6 * 15 * Nf)               # lift factors, gradient traces
    b["volume"] = vol
    # Interfaces: 3 per element; two trace slots, the area-scaled normal and |n|, the common flux,
    # two gradient-trace slots.
    iface = 3 * Nf * (2 * 5 + 4 + 5 + (2 * 15 if viscous else 0))
    b["iface_flux"] = per_el(iface)
    corr = per_el(5 * Np) + per_el(3 * Nf * 5) + per_el(Np)          # Rpart, common flux, 1/|J|
    corr += per_el(5 * Np) * (4 if mode == "rk" else 1)                # Un, acc r/w, Q write (RK)
    b["correct"] = corr
    return b


def prism_flops_per_point(p: int, viscous: bool = True) -> dict:
    """Per solution point of an all-prism periodic mesh: Nt = N(N+1)/2 triangle nodes x N line
    points per prism, 2 triangular faces of Nt and 3 quadrilateral faces of N^2 flux points."""
    N = p + 1
    Nt = N * (N + 1) // 2
    Np = Nt * N
    fp = 2 * Nt + 3 * N * N                  # face points per prism
    fp_pt = fp / Np
    if_pt = fp_pt / 2
    f = {}
    f["interp_faces"] = (2 * Nt * N + 3 * N * N * Nt) * 5 * 2 / Np
    dense = 2 * Nt + N                        # MACs of one derivative triple (r, s along rows; zeta)
    vol = 2 * 5 * dense                       # divergence with the own-flux correction folded in
    vol += _INVISCID + _TRANSFORM
    if viscous:
        vol += 2 * 5 * dense                  # reference gradient
        vol += 5 * 2 * (3 * N + 2)            # liftings of the 3 quadrilateral and 2 triangular faces
        vol += 5 * 6                          # adding the liftings to the gradient
        vol += fp_pt * 5 * 2                  # jumps at the flux points
        vol += _PHYS_GRAD + _VISCOUS + 30     # + BR2 weights
        vol += (2 * Nt * (15 * (2 * N + 2) + 3 * 2 * N) + 3 * N * N * 15 * 5 * Nt) / Np   # gradient traces
    f["volume"] = vol
    f["iface_flux"] = if_pt * (_RUSANOV + (_VISC_COMMON if viscous else 0))
    f["correct"] = 5 * 2 * (2 + 3 * N) + 5 + 5 * 4
    return f


def point_cost(p: int, viscous: bool = True) -> tuple:
    """(hexahedral, prism) algorithmic flops of one solution point through one stage: the
    per-type costs for fr_partition_cost."""
    return (sum(flops_per_point(p, viscous).values()), sum(prism_flops_per_point(p, viscous).values()))


def prism_bytes_per_point(p: int, viscous: bool = True, mode: str = "rk") -> dict:
    N = p + 1
    Nt = N * (N + 1) // 2
    Np = Nt * N
    fp = 2 * Nt + 3 * N * N
    per_el = lambda doubles: 8.0 * doubles / Np          # noqa: E731
    b = {}
    b["interp_faces"] = per_el(5 * Np) + per_el(5 * fp)
    vol = per_el(5 * Np) + per_el(10 * Np) + per_el(5 * Np)
    if viscous:
        vol += per_el(2 * 5 * fp) + per_el(15 * fp)
    b["volume"] = vol
    b["iface_flux"] = per_el(fp / 2 * (2 * 5 + 4 + 5 + (2 * 15 if viscous else 0)))
    corr = per_el(5 * Np) + per_el(fp / 2 * 5) + per_el(Np)
    corr += per_el(5 * Np) * (4 if mode == "rk" else 1)
    b["correct"] = corr
    return b
