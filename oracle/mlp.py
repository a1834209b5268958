"""Plain FP64 reference of the small network of the learned weights (TEST
INFRASTRUCTURE ONLY: used by tests/ to check the CUDA training kernels).

y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 with x in R^16, two hidden layers of
64, one output; loss = mean over the batch of (y - t)^2.  Gradients by the
chain rule, written out layer by layer.  Parameter vector layout (shared with
the CUDA kernels as data): W1 [64][16], b1 [64], W2 [64][64], b2 [64], W3 [64],
b3 [1] (5313 values).

`rnd`, when given, is applied to both operands of every matrix product (the
two hidden-layer products forward; the weight-gradient and back-propagation
products of those layers backward), so that a test can evaluate the network
with operands rounded to the precision a kernel multiplies in; everything else
stays FP64.  Without it the whole computation is FP64.
"""
from __future__ import annotations

import numpy as np

NI, NH = 16, 64
SIZES = [("W1", (NH, NI)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH,)),
         ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SIZES])


def _id(a):
    return a


def forward(theta: np.ndarray, X: np.ndarray, rnd=None):
    r = rnd or _id
    p = unpack(theta)
    z1 = r(X) @ r(p["W1"]).T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = r(h1) @ r(p["W2"]).T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"] + p["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss(theta: np.ndarray, X: np.ndarray, t: np.ndarray) -> float:
    y, _ = forward(theta, X)
    return float(np.mean((y - t) ** 2))


def backward(theta: np.ndarray, X: np.ndarray, dy: np.ndarray, rnd=None) -> np.ndarray:
    """Gradient of sum_i dy_i y_i(theta): back-propagation of per-sample upstream
    gradients dy through the network."""
    r = rnd or _id
    p = unpack(theta)
    y, (X, z1, h1, z2, h2) = forward(theta, X, rnd)
    g = {"W3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, p["W3"]) * (z2 > 0)
    g["W2"] = r(dz2).T @ r(h1)
    g["b2"] = dz2.sum(axis=0)
    dz1 = (r(dz2) @ r(p["W2"])) * (z1 > 0)
    g["W1"] = r(dz1).T @ r(X)
    g["b1"] = dz1.sum(axis=0)
    return pack(g)


def grad(theta: np.ndarray, X: np.ndarray, t: np.ndarray, rnd=None) -> np.ndarray:
    """Gradient of the mean squared error: dL/dy = 2 (y - t) / B, back-propagated."""
    y, _ = forward(theta, X, rnd)
    return backward(theta, X, 2.0 * (y - t) / len(t), rnd)


def init(seed: int) -> np.ndarray:
    """He-scaled normal weights, zero biases."""
    rng = np.random.default_rng(seed)
    p = {"W1": rng.standard_normal((NH, NI)) * np.sqrt(2.0 / NI), "b1": np.zeros(NH),
         "W2": rng.standard_normal((NH, NH)) * np.sqrt(2.0 / NH), "b2": np.zeros(NH),
         "W3": rng.standard_normal(NH) * np.sqrt(1.0 / NH), "b3": np.zeros(1)}
    return pack(p)
