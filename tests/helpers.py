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
