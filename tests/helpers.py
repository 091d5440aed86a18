"""Shared test utilities: parity metrics and library bootstrap."""
import os

import numpy as np

from paper_2308_06605_gb300 import build as B
from paper_2308_06605_gb300 import fr


def ensure_lib():
    if not os.path.exists(fr.LIB_PATH):
        B.build()
    return fr.load()


def parity_error(got, want, floor=1e-3):
    """Per-entry error |got - want| / max(|want|, s_v) with s_v = floor * max_mesh |want_v|.

    Returns the maximum over entries per variable (last axis).  A relative bound per residual
    entry, with a per-variable floor for entries near zero.
    """
    got = np.asarray(got).reshape(-1, 5)
    want = np.asarray(want).reshape(-1, 5)
    s = floor * np.abs(want).max(axis=0)
    den = np.maximum(np.abs(want), s[None, :])
    den = np.where(den > 0, den, 1.0)
    return (np.abs(got - want) / den).max(axis=0)


def assert_parity(got, want, rel=1e-12, floor=1e-3):
    err = parity_error(got, want, floor)
    assert np.all(err <= rel), f"per-variable max relative error {err} > {rel}"
    return err


def assert_residual_parity(got, want, scale, rel=1e-12):
    """Residual parity per entry: |got - want| <= rel * S, S = the entry's magnitude scale from
    the oracle (sum of the magnitudes of the terms whose sum is the entry, Eq. 3).  Any two
    FP64 evaluation orders differ by a few ulps of S; an entry that is small because its terms
    cancel cannot be reproduced to 1e-12 of itself."""
    got = np.asarray(got)
    want = np.asarray(want)
    scale = np.asarray(scale)
    err = (np.abs(got - want) / scale).reshape(-1, 5).max(axis=0)
    norm = (np.abs(got - want).reshape(-1, 5).max(axis=0) / np.abs(want).reshape(-1, 5).max(axis=0))
    assert np.all(err <= rel), f"per-entry error / magnitude scale {err} > {rel} (normwise {norm})"
    return err


def assert_state_parity(got, want, scale, elapsed, rel=1e-12):
    """State parity after RK steps: |got - want| <= rel * (|want| + elapsed * S), i.e. the
    residual bar integrated over the elapsed time (S = magnitude scale of the initial residual)."""
    den = np.abs(want) + elapsed * np.asarray(scale)
    err = (np.abs(np.asarray(got) - want) / den).reshape(-1, 5).max(axis=0)
    assert np.all(err <= rel), f"state error {err} > {rel}"
    return err


def vcjh_c(p, which):
    """Members of the energy-stable correction family (Vincent, Castonguay & Jameson 2011) at
    degree p: dg (c = 0), sd (c_SD = 2p / ((2p+1)(p+1)(a_p p!)^2)), hu (c_HU = 2(p+1) /
    ((2p+1) p (a_p p!)^2)), neg (half the lower limit c_- = -2 / ((2p+1)(a_p p!)^2)), big (10 c_HU);
    a_p p! = (2p)! / (2^p p!)."""
    import math
    apf = math.factorial(2 * p) / (2.0 ** p * math.factorial(p))
    if which == "dg":
        return 0.0
    if which == "sd":
        return 2.0 * p / ((2 * p + 1) * (p + 1) * apf ** 2)
    if which == "hu":
        return 2.0 * (p + 1) / ((2 * p + 1) * p * apf ** 2)
    if which == "neg":
        return -1.0 / ((2 * p + 1) * apf ** 2)
    if which == "big":
        return 10.0 * vcjh_c(p, "hu")
    raise ValueError(which)


def load_g13_reference():
    """The 40-digit low-Mach residual fixture (tests/golden/g13_tgv_ma01_reference.txt):
    {(p, n1): (Q [n1][N^3][5], R [n1][N^3][5])}."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "g13_tgv_ma01_reference.txt")
    rows = np.loadtxt(path, comments="#")
    out = {}
    for p, n1 in sorted({(int(r[0]), int(r[1])) for r in rows}):
        sel = rows[(rows[:, 0] == p) & (rows[:, 1] == n1)]
        Np = (p + 1) ** 3
        Q = np.zeros((n1, Np, 5))
        R = np.zeros((n1, Np, 5))
        for r in sel:
            e, m = int(r[2]), int(r[3])
            Q[e, m] = r[4:9]
            R[e, m] = r[9:14]
        out[(p, n1)] = (Q, R)
    return out
