"""Writes `g13_tgv_ma01_reference.txt`: the hexahedral Navier-Stokes residual of a low-Mach
Taylor-Green state computed at 40 significant digits by `oracle.weakdg_mp` (the independent
weak-form DG restatement of section "FR Algorithm", Eq. 3), with the state it was computed on.

Cases: periodic boxes [0, 2pi]^3 of n1 x 1 x 1 elements, (p, n1) = (2, 2) and (3, 1); Taylor-Green
vortex at Ma 0.1, Re 1600 (gamma 1.4, Pr 0.71, BR2 with eta = 6), random-phase perturbation 1e-3
with seed 3.  At Ma 0.1 the energy entries of the residual are sums of terms of size ~250 / h that
cancel to O(1e-2 .. 1) or less, which is what the per-entry tolerance of the parity tests is about.

Run from the repository root:  python tests/golden/make_g13_reference.py
Only `oracle/` and the seeded input generators are used.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle.hexfr import HexFR  # noqa: E402
from oracle.weakdg_mp import brute_force_residual  # noqa: E402
from paper_2308_06605_gb300 import inputs as I  # noqa: E402

CASES = [(2, 2), (3, 1)]
OUT = os.path.join(HERE, "g13_tgv_ma01_reference.txt")


def case_setup(p, n1):
    """Mesh, physics and state of one case (also used by the tests that read the file)."""
    L = 2 * np.pi
    desc = I.hex_box_mesh((n1, 1, 1), lo=(0.0, 0.0, 0.0), hi=(L, L, L))
    phys = I.tgv_physics(Ma=0.1, Re=1600.0)
    return desc, phys


def main():
    lines = ["# Residual dQ/dt of low-Mach Taylor-Green states at 40 digits (oracle.weakdg_mp), written by",
             "# tests/golden/make_g13_reference.py.  Per line: p n1 e m  Q_0..Q_4 (the state, repr)",
             "# R_0..R_4 (the 40-digit residual rounded to float64, printed with 21 digits)."]
    for p, n1 in CASES:
        desc, phys = case_setup(p, n1)
        x = HexFR(desc, phys, p).x
        Q = I.tgv_state(x, Ma=0.1, perturb=1e-3, seed=3)
        L = 2 * np.pi
        R = brute_force_residual(Q, p, n1, [[1, 0, 0], [0, 1, 0], [0, 0, 1]], (L / n1, L, L), phys.gamma,
                                 phys.R, phys.mu, phys.Pr, 6, True)
        for e in range(n1):
            for m in range(Q.shape[1]):
                q = " ".join(repr(float(v)) for v in Q[e, m])
                r = " ".join(f"{v:.20e}" for v in R[e, m])
                lines.append(f"{p} {n1} {e} {m} {q} {r}")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
