"""Host-side pieces of the closure pipeline: filtering and targets (CPU only)."""
import numpy as np

from paper_2308_06605_gb300 import closure as CL


def test_filter_is_projection():
    F = CL.filter_1d(5, 2)
    x, _ = np.polynomial.legendre.leggauss(6)
    xc, _ = np.polynomial.legendre.leggauss(3)
    for k in range(3):                                   # degree <= 2 passes unchanged
        np.testing.assert_allclose(F @ x ** k, xc ** k, atol=1e-13)
    # degree 3 and 4 Legendre modes are removed
    for k in (3, 4):
        np.testing.assert_allclose(F @ np.polynomial.legendre.legval(x, np.eye(6)[k]), 0, atol=1e-13)
    F3 = CL.filter_3d(4, 2)
    np.testing.assert_allclose(F3 @ np.ones(125), np.ones(27), atol=1e-13)     # constants preserved


def test_targets_vanish_for_resolved_fields_and_gradient_is_exact():
    p_f, p_c, h = 4, 2, 0.5
    x, _ = np.polynomial.legendre.leggauss(p_f + 1)
    X = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1)[..., ::-1].reshape(-1, 3) * h / 2   # (x, y, z)
    A = np.array([[0.2, -0.1, 0.3], [0.0, 0.4, 0.1], [-0.2, 0.3, -0.6]])
    u = X @ A.T                                          # linear velocity: u_i u_j is degree 2
    Q = np.concatenate([np.ones((125, 1)), u, np.full((125, 1), 3.0)], axis=1)[None]
    feats, nu, Pi, SS = CL.features_targets(Q, h, p_f, p_c, with_transfer=True)
    np.testing.assert_allclose(feats[0, :9], A.ravel(), atol=1e-12)
    S = 0.5 * (A + A.T)
    np.testing.assert_allclose(feats[0, 9], np.sqrt(2 * np.sum(S * S)), rtol=1e-12)
    assert abs(nu[0]) < 1e-12 and abs(Pi[0]) < 1e-12
