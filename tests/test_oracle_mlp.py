"""Pins of the oracle MLP closure: activations and the backpropagated gradient (CPU only)."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_activation_closed_forms():
    a = np.linspace(-4, 4, 41)
    # gelu(a) = a Phi(a); Phi(0) = 1/2, gelu(-a) = gelu(a) - a
    np.testing.assert_allclose(mlp.gelu(np.array([0.0, 1.0])), [0.0, 0.5 * (1 + math.erf(1 / math.sqrt(2)))])
    np.testing.assert_allclose(mlp.gelu(-a), mlp.gelu(a) - a, atol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_prime(a), (mlp.gelu(a + h) - mlp.gelu(a - h)) / (2 * h), rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(mlp.softplus(np.array([0.0, 50.0, -50.0])), [math.log(2.0), 50.0, math.exp(-50.0)],
                               rtol=1e-15)
    z = np.linspace(-6, 6, 25)
    np.testing.assert_allclose((mlp.softplus(z + h) - mlp.softplus(z - h)) / (2 * h), mlp.sigmoid(z), rtol=1e-8)


def test_parameter_count_and_layout():
    assert mlp.N_PARAMS == 64 * 11 + 64 + 2 * (64 * 64 + 64) + 64 + 1 == 9153
    p = np.arange(mlp.N_PARAMS, dtype=np.float64)
    np.testing.assert_array_equal(mlp.pack(mlp.unpack(p)), p)


@pytest.mark.parametrize("seed", [0, 1])
def test_backprop_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    params = 0.3 * rng.standard_normal(mlp.N_PARAMS)
    X = rng.standard_normal((17, 11))
    y = np.abs(rng.standard_normal(17))
    loss, g = mlp.loss_and_grad(params, X, y)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [mlp.N_PARAMS - 1, 0, 704, 9152 - 64]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(params)
        e[i] = h
        fd = (mlp.loss_and_grad(params + e, X, y)[0] - mlp.loss_and_grad(params - e, X, y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_single_hidden_path_closed_form():
    """With all weights zero except one path x_0 -> h1_0 -> h2_0 -> h3_0 -> z, the output is a
    composition of scalar functions."""
    d = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    d["W1"][0, 0], d["W2"][0, 0], d["W3"][0, 0], d["w4"][0], d["b4"][0] = 1.5, -0.7, 2.0, 0.9, 0.1
    x = np.zeros((1, 11))
    x[0, 0] = 0.8
    nu, _ = mlp.forward(mlp.pack(d), x)
    g = lambda v: 0.5 * v * (1 + math.erf(v / math.sqrt(2)))  # noqa: E731
    # Zero-weight neurons give gelu(0) = 0, so only the one path contributes.
    z = 0.9 * g(2.0 * g(-0.7 * g(1.5 * 0.8))) + 0.1
    assert abs(nu[0] - math.log1p(math.exp(z))) < 1e-15


def _constant_closure(z0, s_out=2.0):
    d = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    d["b4"][0] = z0
    scales = (np.zeros(11), np.ones(11), s_out)
    return mlp.pack(d), scales


def test_closure_equals_plain_ns_with_effective_viscosity():
    """Constant network output and uniform density: nu_t is one number on a uniform mesh, so the
    closure residual equals the plain residual with mu' = mu + nu_t and Pr' = mu' cp / kappa'."""
    from paper_2308_06605_gb300 import inputs as I
    from oracle.hexfr import HexFR, PR_TURB
    d = I.hex_box_mesh((3, 3, 3), seed=2, rotate=True, shuffle=True)
    ph = I.Physics(gamma=1.4, R=1.0, mu=0.01, Pr=0.71, viscous=1)
    m = HexFR(d, ph, 2)
    X = m.x
    Q = I.conserved(np.ones(X.shape[:2]), 0.2 * np.sin(X[..., 1]), 0.1 * np.cos(X[..., 2]), 0.05 * np.sin(X[..., 0]),
                    1.0 + 0.1 * np.cos(X[..., 0] + X[..., 1]), 1.4)
    params, scales = _constant_closure(0.3)
    m.set_closure(params, scales)
    R_cl = m.residual(Q)
    nu = scales[2] * (m.h[0] / 3) ** 2 * math.log1p(math.exp(0.3))
    np.testing.assert_allclose(m.last_nu, nu, rtol=1e-13)
    cp = 1.4 / 0.4
    mu2 = 0.01 + nu
    kap2 = 0.01 * cp / 0.71 + nu * cp / PR_TURB
    m2 = HexFR(d, I.Physics(gamma=1.4, R=1.0, mu=mu2, Pr=mu2 * cp / kap2, viscous=1), 2)
    R_ref = m2.residual(Q)
    np.testing.assert_allclose(R_cl, R_ref, rtol=0, atol=1e-12 * np.abs(R_ref).max())


def test_closure_element_mean_gradient_and_conservation():
    from paper_2308_06605_gb300 import inputs as I
    from oracle.hexfr import HexFR
    d = I.hex_box_mesh((3, 3, 3), hi=(1.0, 1.0, 1.0), periodic=(False, False, False),
                       wall_tags={t: (I.BC_DIRICHLET, (1.0, 0.0, 0.0, 0.0, 2.5)) for t in range(1, 7)}, seed=1, rotate=True)
    ph = I.Physics(gamma=1.4, R=1.0, mu=0.01, Pr=0.71, viscous=1)
    m = HexFR(d, ph, 2)
    X = m.x
    A = np.array([[0.3, -0.2, 0.1], [0.05, 0.4, -0.3], [0.2, 0.1, -0.7]])
    u = X @ A.T                                      # linear velocity: exact gradient A everywhere
    Q = I.conserved(np.ones(X.shape[:2]), u[..., 0], u[..., 1], u[..., 2], np.full(X.shape[:2], 1.0), 1.4)
    rng = np.random.default_rng(3)
    params = 0.2 * rng.standard_normal(mlp.N_PARAMS)
    scales = (np.zeros(11), np.ones(11), 1.0)
    m.set_closure(params, scales)
    m.residual(Q)
    # The element away from the boundary sees no jumps: its corrected gradient is exactly A.
    centre = np.argmin(np.linalg.norm(m.x.mean(axis=1) - 0.5, axis=1))
    Xf = mlp.features(np.broadcast_to(A, (m.E, 3, 3)), m.h, 2)
    np.testing.assert_allclose(m.last_nu[centre], mlp.eddy_viscosity(params, scales, Xf)[centre], rtol=1e-10)
    assert np.all(m.last_nu >= 0)
    # conservation on a periodic mesh with the closure on
    dp = I.hex_box_mesh((3, 3, 3), seed=4, perturb=0.1, rotate=True)
    mp_ = HexFR(dp, ph, 2)
    mp_.set_closure(params, scales)
    Qp = I.tgv_state(mp_.x, Ma=0.3, perturb=1e-2)
    R = mp_.residual(Qp)
    s = np.abs(mp_.integrate(R))
    a = np.einsum('m,em,emv->v', mp_.W, mp_.detJ, np.abs(R))
    assert np.all(s <= 1e-12 * a)
