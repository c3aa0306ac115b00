"""Oracle of the learned detection threshold -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
import this module; the product path never does.

The paper verifies a checksum by comparing the residual with "a
predetermined threshold" and leaves its value open (Section 2.2).  The
library's analytic threshold is tau = lambda * u * (norm product) with a
fixed lambda.  The learned threshold replaces the constant lambda of a tile
by lambda_t = scale * 2^f(x_t), where f is a 5 -> 32 -> 32 -> 1 ReLU network
of cheap tile features x_t, trained on the GPU to predict
log2(lambda_needed), the smallest lambda at which the fault-free tile would
have raised no flag.  Nothing of this is in the paper; this module is the
plain float64 definition the GPU kernels are checked against:

  * the parameter layout (one flat vector, the order the kernels read),
  * the tile features,
  * forward pass, mean-squared-error loss and its gradient by backprop,
  * Adam (Kingma & Ba, 2015) with bias correction.

Written for reading, not speed: numpy matrix products are the only
library steps.
"""
from __future__ import annotations

import numpy as np

N_IN = 5
N_H = 32
# flat parameter vector: W1 [N_H][N_IN], b1 [N_H], W2 [N_H][N_H], b2 [N_H],
# W3 [N_H], b3 [1]
SHAPES = (("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_H,)), ("b3", (1,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)  # 1281

DTYPE_CODE = {"f32": 0.0, "bf16": 1.0, "e4m3": 2.0}


def unpack(theta: np.ndarray) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (N_PARAMS,)
    out, at = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[at:at + n].reshape(shape)
        at += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def features(K: int, rows: int, cols: int, co_a: float, co_b: float, dtype: str) -> np.ndarray:
    """The 5 inputs of a tile: log2 K / 16; the coherence of A's row block,
    ||e^T A_I||_2 / (sqrt(|I|) ||A_I||_F) in [0, 1]; the same of B's column
    block, ||B_J e||_2 / (sqrt(|J|) ||B_J||_F); the operand type (0 fp32,
    0.5 bf16, 1 e4m3); log2(|I| |J|) / 16.  The checksum residual of a tile
    scales with its data, so no absolute norm enters."""
    return np.array([np.log2(K) / 16.0, co_a, co_b, DTYPE_CODE[dtype] / 2.0,
                     np.log2(rows * cols) / 16.0], dtype=np.float64)


def coherence(block: np.ndarray, axis: int) -> float:
    """||sum of the block along `axis`||_2 / (sqrt(count) ||block||_F): 1 when
    all rows (axis 0) or columns (axis 1) are equal, about count^-1/2 for
    independent zero-mean ones, 0 for an all-zero block."""
    block = np.asarray(block, dtype=np.float64)
    fro = np.sqrt(np.sum(block * block))
    if fro == 0.0:
        return 0.0
    s = block.sum(axis=axis)
    return float(np.sqrt(np.sum(s * s)) / (np.sqrt(block.shape[axis]) * fro))


def forward(theta: np.ndarray, X: np.ndarray):
    """y = W3 . relu(W2 relu(W1 x + b1) + b2) + b3 for each row x of X.
    Returns y [n] and the cache the backward pass needs."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"] + p["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss(theta: np.ndarray, X: np.ndarray, t: np.ndarray) -> float:
    """Mean squared error of the predictions against the targets t."""
    y, _ = forward(theta, X)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def grad(theta: np.ndarray, X: np.ndarray, t: np.ndarray):
    """(loss, d loss / d theta) by the chain rule, layer by layer.  ReLU'(z)
    is taken as 1 for z > 0 and 0 otherwise."""
    p = unpack(theta)
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    t = np.asarray(t, dtype=np.float64)
    n = X.shape[0]
    dy = 2.0 * (y - t) / n                      # d loss / d y
    g = {"W3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dh2 = np.outer(dy, p["W3"])
    dz2 = dh2 * (z2 > 0.0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (z1 > 0.0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return float(np.mean((y - t) ** 2)), pack(g)


def adam_step(theta, g, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update at 1-based `step`: first and second moment estimates,
    bias-corrected, then theta -= lr * m_hat / (sqrt(v_hat) + eps)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    theta = theta - lr * m_hat / (np.sqrt(v_hat) + eps)
    return theta, m, v


def train(theta0, X, t, epochs: int, batch: int, lr: float):
    """Minibatch Adam over the rows of X in their given order, batch after
    batch (the last one may be short), `epochs` times.  Returns the trained
    parameters and the loss of every step."""
    theta = np.asarray(theta0, dtype=np.float64).copy()
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    n = X.shape[0]
    losses, step = [], 0
    for _ in range(epochs):
        for s in range(0, n, batch):
            step += 1
            L, g = grad(theta, X[s:s + batch], t[s:s + batch])
            theta, m, v = adam_step(theta, g, m, v, step, lr)
            losses.append(L)
    return theta, losses
