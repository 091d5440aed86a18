"""Closure network on the GPU vs the FP64 oracle (marked gpu).

Training kernels (FP32): loss and every gradient vs oracle.mlp (FP64) within FP32 bounds
(loss 1e-5 relative, gradients 1e-4 of the largest component); one Adam step vs its closed form.
Inference inside the residual (BF16 weights, FP32 activations): nu_t per element vs the oracle
evaluated with the same BF16-rounded weights, 1e-5 relative; residual 1e-6 of the magnitude scale.
"""
import numpy as np
import pytest

from paper_2308_06605_gb300 import fr
from paper_2308_06605_gb300 import inputs as I
from oracle import mlp
from oracle.hexfr import HexFR

from helpers import assert_residual_parity, ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def bf16_round(a):
    """Round float32 values to bfloat16 (round to nearest even) and back."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (u.astype(np.uint32) << 16).view(np.float32)


def _random_net(seed, scale=0.25):
    rng = np.random.default_rng(seed)
    return (scale * rng.standard_normal(mlp.N_PARAMS)).astype(np.float32)


def test_training_kernels_match_oracle():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    n = 300
    X = (rng.standard_normal((n, 11)) * np.linspace(0.5, 3, 11) + np.linspace(-1, 1, 11)).astype(np.float32)
    y = np.abs(rng.standard_normal(n)).astype(np.float32)
    scales = np.concatenate([X.mean(0), X.std(0), [1.0]]).astype(np.float32)
    P = _random_net(1)
    tr = fr.MLPTrainer(P, scales, max_batch=n)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    loss, g = tr.loss_grad(Xd, yd)
    torch.cuda.synchronize()
    Xn = (X.astype(np.float64) - scales[:11].astype(np.float64)) / scales[11:22].astype(np.float64)
    lo, go = mlp.loss_and_grad(P.astype(np.float64), Xn, y.astype(np.float64))
    assert abs(float(loss.item()) - lo) <= 1e-5 * lo
    gg = g.cpu().numpy().astype(np.float64)
    assert np.abs(gg - go).max() <= 1e-4 * np.abs(go).max()
    assert np.linalg.norm(gg - go) <= 1e-5 * np.linalg.norm(go) * 10
    out = tr.forward(Xd).cpu().numpy()
    nu_o, _ = mlp.forward(P.astype(np.float64), Xn)
    np.testing.assert_allclose(out, nu_o, rtol=1e-5, atol=1e-6)
    # One Adam step: m = (1-b1) g, v = (1-b2) g^2, P -= lr (m/(1-b1)) / (sqrt(v/(1-b2)) + eps)
    lr, eps = 1e-3, 1e-8
    tr.adam(lr, 0.9, 0.999, eps)
    want = P.astype(np.float64) - lr * gg / (np.abs(gg) + eps)
    np.testing.assert_allclose(tr.P.cpu().numpy(), want, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("precision", [0, 1])
def test_closure_inference_in_residual(precision):
    d = I.hex_box_mesh((3, 3, 3), seed=5, rotate=True, shuffle=True, perturb=0.05)
    phys = I.tgv_physics(Ma=0.2, Re=300.0)
    phys.precision = precision
    ora = HexFR(d, phys, 2)
    Q = np.ascontiguousarray(I.tgv_state(ora.x, Ma=0.2, perturb=2e-2, seed=1))
    P = _random_net(2)
    feats_scale = np.array([1.0] * 9 + [1.5, 0.2], dtype=np.float32)
    scales = np.concatenate([np.zeros(11, np.float32), feats_scale, np.float32([0.8])]).astype(np.float32)
    with fr.Mesh(d, phys, 2) as g:
        g.set_closure(P, scales)
        g.set_state(Q)
        R = g.residual()
        nu_g = g.closure_nu()
    ora.set_closure(bf16_round(P).astype(np.float64),
                    (scales[:11].astype(np.float64), scales[11:22].astype(np.float64), float(scales[22])))
    Ro = ora.residual(Q)
    assert np.all(ora.last_nu > 0)
    np.testing.assert_allclose(nu_g, ora.last_nu, rtol=1e-5)
    assert_residual_parity(R, Ro, ora.residual(Q, magnitude=True), rel=1e-6)
