"""FP64 oracle of the learned surrogate (a per-material MLP standing in for a cacheable
node's UV-only sub-graph).

TEST INFRASTRUCTURE ONLY (see oracle/pmc_oracle.h).  Plain numpy in float64; matrix
products are the only library routine used.

Network (the definition the CUDA kernels implement):
  features  g(u, v) = [sin pi k u]_{k=1..16}, [cos pi k u]_{k=1..16},
                      [sin pi k v]_{k=1..16}, [cos pi k v]_{k=1..16}          (64)
            (half-range frequencies: a function of g need not repeat from u = 0 to 1)
  h1 = relu(g W1 + b1)   (64)      h2 = relu(h1 W2 + b2)   (64)      y = h2 W3 + b3   (3)
  loss = mean over points and channels of (y - t)^2
Parameters are one flat vector of 8,515 values in the order
  W1 [64 in][64 out], b1 [64], W2 [64][64], b2 [64], W3 [64][3], b3 [3].
Optimiser: Adam (Kingma & Ba 2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

N_FREQ = 16
N_FEAT = 4 * N_FREQ
N_HID = 64
N_OUT = 3
SHAPES = (("W1", (N_FEAT, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID, N_OUT)), ("b3", (N_OUT,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
assert N_PARAMS == 8515


def unpack(theta):
    """Flat parameter vector -> dict of arrays (views)."""
    theta = np.asarray(theta, dtype=np.float64)
    out, k = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = theta[k:k + size].reshape(shape)
        k += size
    return out


def pack(params) -> np.ndarray:
    return np.concatenate([np.asarray(params[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def features(u, v) -> np.ndarray:
    """Fourier features of (u, v): (n, 64)."""
    u = np.asarray(u, dtype=np.float64)[:, None]
    v = np.asarray(v, dtype=np.float64)[:, None]
    k = np.arange(1, N_FREQ + 1, dtype=np.float64)[None, :]
    return np.concatenate([np.sin(np.pi * k * u), np.cos(np.pi * k * u),
                           np.sin(np.pi * k * v), np.cos(np.pi * k * v)], axis=1)


def forward(theta, g):
    """Returns y (n, 3) and the activations needed by backward."""
    p = unpack(theta)
    z1 = g @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"] + p["b3"]
    return y, (g, z1, h1, z2, h2)


def loss(theta, g, t) -> float:
    y, _ = forward(theta, g)
    return float(np.mean((y - t) ** 2))


def gradient(theta, g, t):
    """Loss and its gradient with respect to the flat parameters (backpropagation)."""
    p = unpack(theta)
    y, (g, z1, h1, z2, h2) = forward(theta, g)
    n = g.shape[0]
    dy = 2.0 * (y - t) / (n * N_OUT)
    grads = {"W3": h2.T @ dy, "b3": dy.sum(axis=0)}
    dh2 = (dy @ p["W3"].T) * (z2 > 0)
    grads["W2"] = h1.T @ dh2
    grads["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ p["W2"].T) * (z1 > 0)
    grads["W1"] = g.T @ dh1
    grads["b1"] = dh1.sum(axis=0)
    return float(np.mean((y - t) ** 2)), pack(grads)


def adam_step(theta, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    bits = a.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    bits = (bits + 0x7FFF + lsb) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def predict(theta, u, v, clamp=True) -> np.ndarray:
    """Surrogate value of a cacheable node at (u, v): (n, 3), clamped to [0, 1] like the
    node it stands in for."""
    y, _ = forward(theta, features(u, v))
    return np.clip(y, 0.0, 1.0) if clamp else y
