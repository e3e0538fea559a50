"""FP64 oracle of the learned ALS extrapolation network (test infrastructure only).

Network (the extrapolation step proposer): input x in R^40, two hidden layers of width
64 with tanh, one output, step factor alpha = 1 + 3 sigmoid(z) in [1, 4]:
    h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), z = w3 . h2 + b3.
Parameters are packed in this order into one vector: W1 (64 x 40, row-major), b1 (64),
W2 (64 x 64), b2 (64), w3 (64), b3 (1): 6849 numbers.
Training loss: mean squared error between alpha and the target step factor.
Everything here is FP64; the GPU kernels use BF16 copies of the weights with FP32
accumulation and are compared against these functions.
"""
from __future__ import annotations

import numpy as np

NIN, NH = 40, 64
SIZES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)),
         ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SIZES])


def forward(theta, X):
    """alpha (n,) and the intermediates for backward; X is (n, 40)."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    z = h2 @ p["w3"] + p["b3"][0]
    s = 1.0 / (1.0 + np.exp(-z))
    alpha = 1.0 + 3.0 * s
    return alpha, dict(X=X, h1=h1, h2=h2, z=z, s=s)


def loss_and_grad(theta, X, y):
    """MSE loss (1/n) sum (alpha - y)^2 and its gradient w.r.t. the packed parameters,
    by the chain rule through the layers above (reverse order)."""
    p = unpack(theta)
    alpha, c = forward(theta, X)
    n = alpha.shape[0]
    r = alpha - np.asarray(y, dtype=np.float64)
    loss = float(np.mean(r * r))
    dalpha = 2.0 * r / n
    dz = dalpha * 3.0 * c["s"] * (1.0 - c["s"])
    g = {"w3": c["h2"].T @ dz, "b3": np.array([dz.sum()])}
    da2 = np.outer(dz, p["w3"]) * (1.0 - c["h2"] ** 2)
    g["W2"] = da2.T @ c["h1"]
    g["b2"] = da2.sum(axis=0)
    da1 = (da2 @ p["W2"]) * (1.0 - c["h1"] ** 2)
    g["W1"] = da1.T @ c["X"]
    g["b1"] = da1.sum(axis=0)
    return loss, pack(g)


def init(seed):
    """Glorot-uniform weights, zero biases, from numpy PCG64 (the GPU side draws its own
    initialisation; this is for the oracle's tests)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SIZES:
        if name.startswith("W") or name == "w3":
            fan_in = shape[-1] if len(shape) == 2 else NH
            fan_out = shape[0] if len(shape) == 2 else 1
            lim = np.sqrt(6.0 / (fan_in + fan_out))
            p[name] = rng.uniform(-lim, lim, shape)
        else:
            p[name] = np.zeros(shape)
    return pack(p)


def adam_step(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ---- features of the ALS history (the network's input) --------------------------------
def features(loss_hist, change_hist):
    """40 inputs from the last 8 sweeps, most recent first, zero-padded:
    8 values log10(max(log(L_{s-1}) - log(L_s), 1e-12)) / 6 and, per sweep, the four
    per-mode values log10(max(||B_k^s - B_k^{s-1}|| / ||B_k^s||, 1e-12)) / 6 (B = factors
    with lam absorbed into the last mode). loss_hist: losses L_0..L_s (at least 1);
    change_hist: list of 4-vectors, one per sweep."""
    f = np.zeros(40)
    L = np.asarray(loss_hist, dtype=np.float64)
    for i in range(8):
        s = len(L) - 1 - i
        if s >= 1:
            d = np.log(L[s - 1]) - np.log(L[s])
            f[i] = np.log10(max(d, 1e-12)) / 6.0
    for i in range(8):
        s = len(change_hist) - 1 - i
        if s >= 0:
            f[8 + 4 * i: 12 + 4 * i] = np.log10(np.maximum(np.asarray(change_hist[s]), 1e-12)) / 6.0
    return f
