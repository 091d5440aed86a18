"""FP64 reference of the eddy-viscosity MLP closure (oracle; test infrastructure only).

The paper lists LES sub-grid-scale models among its physical models (section "FR Algorithm",
code overview) without specifying one; this build's closure is a small network predicting a
non-negative eddy viscosity per element:

  x (11) = element-mean velocity gradient du_i/dx_j (9, row-major), |S| = sqrt(2 S_ij S_ij) of that
           gradient, and Delta = h / (p + 1)
  x^ = (x - mean) / std                      (normalisation constants shipped with the weights)
  h1 = gelu(W1 x^ + b1), h2 = gelu(W2 h1 + b2), h3 = gelu(W3 h2 + b3)     (64 each)
  z = w4 . h3 + b4,   nu^ = softplus(z),   nu_t = s_out * Delta^2 * nu^
with gelu(a) = a Phi(a) (Phi the standard normal CDF, via erf) and softplus(z) = log(1 + e^z).
Training minimises the mean squared error of nu^ against the target nu_t / (s_out Delta^2).

Flat parameter layout (float32 on the device, float64 here): W1[64][11], b1[64], W2[64][64],
b2[64], W3[64][64], b3[64], w4[64], b4[1] -- 9153 values.
"""
from __future__ import annotations

import math

import numpy as np

NIN, NH = 11, 64
SHAPES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH, NH)), ("b3", (NH,)),
          ("w4", (NH,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)

_erf = np.vectorize(math.erf)


def unpack(params):
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(params[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def gelu(a):
    return 0.5 * a * (1.0 + _erf(a / math.sqrt(2.0)))


def gelu_prime(a):
    return 0.5 * (1.0 + _erf(a / math.sqrt(2.0))) + a * np.exp(-0.5 * a * a) / math.sqrt(2.0 * math.pi)


def softplus(z):
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(params, Xn):
    """Xn [n][11] normalised inputs -> (nu^ [n], cache)."""
    P = unpack(params)
    a1 = Xn @ P["W1"].T + P["b1"]
    h1 = gelu(a1)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = gelu(a2)
    a3 = h2 @ P["W3"].T + P["b3"]
    h3 = gelu(a3)
    z = h3 @ P["w4"] + P["b4"][0]
    return softplus(z), (Xn, a1, h1, a2, h2, a3, h3, z)


def loss_and_grad(params, Xn, y):
    """Mean squared error of nu^ against y and its gradient with respect to the flat parameters
    (backpropagation written out layer by layer)."""
    P = unpack(params)
    nu, (x, a1, h1, a2, h2, a3, h3, z) = forward(params, Xn)
    n = x.shape[0]
    r = nu - y
    loss = float(np.mean(r * r))
    dz = 2.0 * r * sigmoid(z) / n                    # d loss / d z
    g = {"w4": h3.T @ dz, "b4": np.array([dz.sum()])}
    da3 = np.outer(dz, P["w4"]) * gelu_prime(a3)
    g["W3"], g["b3"] = da3.T @ h2, da3.sum(axis=0)
    da2 = (da3 @ P["W3"]) * gelu_prime(a2)
    g["W2"], g["b2"] = da2.T @ h1, da2.sum(axis=0)
    da1 = (da2 @ P["W2"]) * gelu_prime(a1)
    g["W1"], g["b1"] = da1.T @ x, da1.sum(axis=0)
    return loss, pack(g)


def features(grad_u, h, p):
    """[n][3][3] velocity gradients (du_i/dx_j), element sizes h and order p -> [n][11]."""
    S = 0.5 * (grad_u + np.swapaxes(grad_u, 1, 2))
    Smag = np.sqrt(2.0 * np.sum(S * S, axis=(1, 2)))
    delta = np.broadcast_to(np.asarray(h, dtype=np.float64) / (p + 1), Smag.shape)
    return np.concatenate([grad_u.reshape(-1, 9), Smag[:, None], delta[:, None]], axis=1)


def eddy_viscosity(params, scales, X):
    """nu_t for raw features X [n][11]; scales = (mean[11], std[11], s_out)."""
    mean, std, s_out = scales
    nu, _ = forward(params, (X - mean) / std)
    return s_out * X[:, 10] ** 2 * nu
