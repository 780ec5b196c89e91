"""CPU oracle of the link-travel-time surrogate MLP (float64, numpy).

TEST INFRASTRUCTURE ONLY: the GPU surrogate kernels are checked against it.

The network maps a feature vector of one (link, 15-minute bin) to the link's
travel time: inputs (padded to 64 columns) -> 256 -> 256 -> 256 -> 1 with
GELU after each hidden layer, GELU(x) = x * Phi(x) = 0.5 x (1 + erf(x/sqrt 2))
(Hendrycks and Gimpel 2016), mean-squared-error loss, and Adam updates
(Kingma and Ba 2015, Algorithm 1).  Weights W_l are stored out x in
(row l of W is the weight vector of output unit l).

Every function takes the weights and inputs as given (the GPU keeps BF16
copies of weights and activations; the tests round to BF16 before calling
these and compare against the GPU within a BF16-derived tolerance).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)

DIMS = (64, 256, 256, 256, 1)  # padded input width, three hidden layers, output


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / SQRT2))


def gelu_grad(x):
    """d/dx [x Phi(x)] = Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + erf(x / SQRT2)) + x * INV_SQRT_2PI * np.exp(-0.5 * x * x)


def init_params(seed: int, dims=DIMS, n_in: int = 9) -> dict:
    """He-style initialisation; columns of the first layer beyond the n_in
    real features are zero (they multiply the zero padding)."""
    rng = np.random.default_rng(seed)
    p = {}
    for l in range(len(dims) - 1):
        fan_in = n_in if l == 0 else dims[l]
        w = rng.standard_normal((dims[l + 1], dims[l])) * math.sqrt(2.0 / fan_in)
        if l == 0:
            w[:, n_in:] = 0.0
        p[f"W{l + 1}"] = w
        p[f"b{l + 1}"] = np.zeros(dims[l + 1])
    return p


def forward(p: dict, X: np.ndarray, keep: bool = False, act_round=None):
    """Returns the output y (n,) and, if keep, the pre-activations Z_l and
    activations H_l (H_0 = X).  act_round (optional) is applied to every
    hidden activation, e.g. bf16_round for a network that stores its
    activations in BF16."""
    H = [np.asarray(X, dtype=np.float64)]
    Z = []
    n_layers = len([k for k in p if k.startswith("W")])
    for l in range(1, n_layers + 1):
        z = H[-1] @ p[f"W{l}"].T + p[f"b{l}"]
        Z.append(z)
        if l < n_layers:
            h = gelu(z)
            H.append(act_round(h) if act_round else h)
        else:
            H.append(z)
    y = H[-1][:, 0]
    return (y, Z, H) if keep else y


def loss(p: dict, X, t) -> float:
    y = forward(p, X)
    return float(np.mean((y - t) ** 2))


def backward(p: dict, X, t, act_round=None) -> dict:
    """Gradients of the mean-squared error with respect to every parameter
    (act_round as in forward; the gradient is that of the network with
    rounded activations, taken through the unrounded GELU)."""
    y, Z, H = forward(p, X, keep=True, act_round=act_round)
    n = len(t)
    n_layers = len(Z)
    g = {}
    dz = (2.0 / n) * (y - t)[:, None]           # d loss / d z_last
    for l in range(n_layers, 0, -1):
        g[f"W{l}"] = dz.T @ H[l - 1]
        g[f"b{l}"] = dz.sum(axis=0)
        if l > 1:
            dh = dz @ p[f"W{l}"]
            dz = dh * gelu_grad(Z[l - 2])
    return g


def adam_step(p: dict, g: dict, m: dict, v: dict, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8) -> None:
    """One Adam update in place (Kingma and Ba 2015, Algorithm 1)."""
    for k in p:
        m[k] = beta1 * m[k] + (1 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1 - beta2) * g[k] ** 2
        mh = m[k] / (1 - beta1 ** t)
        vh = v[k] / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
