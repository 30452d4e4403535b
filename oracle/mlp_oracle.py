"""CPU oracle of the learned surrogate: a 4-128-128-128-1 GELU MLP in float64.

TEST INFRASTRUCTURE ONLY (imported by tests/ and the CPU legs of bench.py;
the CUDA engine never imports it). The paper has no learned component; this
module fixes what the engine's hand-written MLP kernels must compute:

  x (4 features) -> h1 = gelu(W1 x + b1) -> h2 = gelu(W2 h1 + b2)
                 -> h3 = gelu(W3 h2 + b3) -> y = w4 . h3 + b4
  gelu(z) = z * Phi(z) = 0.5 z (1 + erf(z / sqrt 2))
  loss = mean over the batch of (y - target)^2

Weights are used rounded to bfloat16 (round to nearest, ties to even, the
format's definition) and everything else is float64, so the engine's FP32
accumulation can be compared with a tolerance. Parameters are one flat
float32 vector in the order W1 (128x4, row-major), b1, W2 (128x128), b2,
W3 (128x128), b3, w4 (128), b4.
"""
from __future__ import annotations

import math

import numpy as np

WIDTH = 128
N_IN = 4
SHAPES = [("W1", (WIDTH, N_IN)), ("b1", (WIDTH,)), ("W2", (WIDTH, WIDTH)), ("b2", (WIDTH,)),
          ("W3", (WIDTH, WIDTH)), ("b3", (WIDTH,)), ("w4", (WIDTH,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)   # 33793


def unflatten(theta):
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[k:k + n], np.float64).reshape(shape)
        k += n
    return out


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even); NaN stays NaN."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32)
    return np.where(np.isnan(f), f, out)


_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(theta, x, bf16=True, keep=False):
    """y (n,) for inputs x (n, 4); with keep, also the pre-activations."""
    p = unflatten(bf16_round(theta) if bf16 else np.asarray(theta, np.float64))
    x = np.asarray(x, np.float64)
    z1 = x @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    z3 = h2 @ p["W3"].T + p["b3"]
    h3 = gelu(z3)
    y = h3 @ p["w4"] + p["b4"][0]
    if keep:
        return y, (x, z1, h1, z2, h2, z3, h3, p)
    return y


def loss_and_grad(theta, x, t, bf16=True):
    """Mean squared error and its gradient with respect to the flat parameters
    (the gradient is taken at the bf16-rounded weights, as the engine does)."""
    y, (x, z1, h1, z2, h2, z3, h3, p) = forward(theta, x, bf16, keep=True)
    n = len(y)
    r = y - np.asarray(t, np.float64)
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    g = {"b4": np.array([dy.sum()]), "w4": h3.T @ dy}
    dz3 = np.outer(dy, p["w4"]) * gelu_grad(z3)
    g["W3"] = dz3.T @ h2
    g["b3"] = dz3.sum(0)
    dz2 = (dz3 @ p["W3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    flat = np.concatenate([g[name].reshape(-1) for name, _ in SHAPES])
    return loss, flat


def adam_step(theta, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba) of float32 master parameters."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    theta = theta - lr * mh / (np.sqrt(vh) + eps)
    return theta.astype(np.float32), m, v
