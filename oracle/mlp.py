"""FP64 numpy oracle of the warm-start network (test infrastructure only).

The network maps 4 inputs to 3 outputs through two tanh hidden layers of 64:
    h1 = tanh(x W1 + b1),  h2 = tanh(h1 W2 + b2),  y = h2 W3 + b3,
with the loss L = mean over samples and outputs of (y - t)^2, trained by
Adam (Kingma & Ba, 2015).  Parameters are one flat vector laid out as
W1 [4][64], b1 [64], W2 [64][64], b2 [64], W3 [64][3], b3 [3] (4675 values),
the layout of the CUDA library's lbm_mlp_* functions.

The paper has no network; this oracle follows the definitions above and is
pinned by central finite differences of the loss (tests).
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 4, 64, 3
SHAPES = [("W1", (N_IN, N_H)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_H, N_OUT)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[k:k + n], dtype=np.float64).reshape(shape)
        k += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel()
                           for name, _ in SHAPES])


def init_params(seed=0):
    """Glorot-uniform weights, zero biases."""
    g = np.random.default_rng(seed)
    parts = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / (shape[0] + shape[1]))
            parts[name] = g.uniform(-lim, lim, shape)
        else:
            parts[name] = np.zeros(shape)
    return pack(parts)


def forward(theta, X):
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ p["W1"] + p["b1"])
    h2 = np.tanh(h1 @ p["W2"] + p["b2"])
    return h2 @ p["W3"] + p["b3"], (X, h1, h2)


def loss(theta, X, T):
    y, _ = forward(theta, X)
    return float(np.mean((y - np.asarray(T, dtype=np.float64)) ** 2))


def gradient(theta, X, T):
    """(loss, dL/dtheta) by back-propagation through the layers above."""
    p = unpack(theta)
    y, (X, h1, h2) = forward(theta, X)
    T = np.asarray(T, dtype=np.float64)
    n = X.shape[0]
    dy = 2.0 * (y - T) / (n * N_OUT)
    g = {"W3": h2.T @ dy, "b3": dy.sum(0)}
    dz2 = (dy @ p["W3"].T) * (1.0 - h2 ** 2)
    g["W2"], g["b2"] = h1.T @ dz2, dz2.sum(0)
    dz1 = (dz2 @ p["W2"].T) * (1.0 - h1 ** 2)
    g["W1"], g["b1"] = X.T @ dz1, dz1.sum(0)
    return float(np.mean((y - T) ** 2)), pack(g)


def adam_train(theta, X, T, order, batch, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam over the given epoch orders (array epochs x n of sample indices);
    minibatch k of an epoch is order[e, k*batch:(k+1)*batch] (a short last
    batch is used as is).  Returns (theta, final minibatch loss)."""
    theta = np.array(theta, dtype=np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    t = 0
    last = None
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    for row in np.asarray(order):
        for k in range(0, len(row), batch):
            idx = row[k:k + batch]
            last, g = gradient(theta, X[idx], T[idx])
            t += 1
            m = beta1 * m + (1 - beta1) * g
            v = beta2 * v + (1 - beta2) * g * g
            mh = m / (1 - beta1 ** t)
            vh = v / (1 - beta2 ** t)
            theta -= lr * mh / (np.sqrt(vh) + eps)
    return theta, last
