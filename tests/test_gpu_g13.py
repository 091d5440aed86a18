"""The GPU residual against the exact (40-digit) residual of low-Mach Taylor-Green states
(tests/golden/g13_tgv_ma01_reference.txt, written from oracle.weakdg_mp): per entry the FP64 path
is within 1e-12 of the entry's magnitude scale S (the sum of the magnitudes of Eq. 3's terms
forming it) and no worse than a small multiple of the FP64 oracle's own error against the same
exact values; the double-float path is within its stated 1e-9 S."""
import numpy as np
import pytest

from oracle.hexfr import HexFR
from paper_2308_06605_gb300 import fr, inputs as I

from helpers import ensure_lib, load_g13_reference

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", [(2, 2), (3, 1)])
def test_gpu_residual_against_40_digit_reference(case):
    ensure_lib()
    p, n1 = case
    Q, Rx = load_g13_reference()[case]
    L = 2 * np.pi
    desc = I.hex_box_mesh((n1, 1, 1), lo=(0.0, 0.0, 0.0), hi=(L, L, L))
    phys = I.tgv_physics(Ma=0.1, Re=1600.0)
    ora = HexFR(desc, phys, p)
    S = ora.residual(Q, magnitude=True)
    ora_err = (np.abs(ora.residual(Q) - Rx) / S).reshape(-1, 5).max(axis=0)
    with fr.Mesh(desc, phys, p) as g:
        g.set_state(Q)
        gpu_err = (np.abs(g.residual() - Rx) / S).reshape(-1, 5).max(axis=0)
    assert np.all(gpu_err <= 1e-12), gpu_err
    assert np.all(gpu_err <= 50 * max(ora_err.max(), 1e-16)), (gpu_err, ora_err)
    phys_m = I.tgv_physics(Ma=0.1, Re=1600.0)
    phys_m.precision = 1
    with fr.Mesh(desc, phys_m, p) as g:
        g.set_state(Q)
        mixed_err = (np.abs(g.residual() - Rx) / S).reshape(-1, 5).max(axis=0)
    assert np.all(mixed_err <= 1e-9), mixed_err
    print(f"p={p}: err/S FP64 GPU {gpu_err.max():.2e}, FP64 oracle {ora_err.max():.2e}, double-float {mixed_err.max():.2e}")
