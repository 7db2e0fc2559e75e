"""FP64 reference of the surrogate MLP's arithmetic (test infrastructure).

A 4 -> 64 -> 64 -> 64 -> 64 -> 2 SiLU network written as plain matrix
products in float64, with BF16 rounding applied exactly where the tensor-core
kernels round (weights, the inputs and activations fed to a layer, SiLU'(z),
and the backward signals fed to a product); sums are FP64. Shares no code
with the CUDA library.
"""
from __future__ import annotations

import numpy as np

H, NIN, NOUT = 64, 4, 2
OUT_SCALE = 4.0
SIZES = [("W1", (H, NIN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)),
         ("b3", (H,)), ("W4", (H, H)), ("b4", (H,)), ("W5", (NOUT, H)), ("b5", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def bf16(x):
    """Round to bfloat16 (nearest, ties to even) through float32, as float64."""
    a = np.asarray(x, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def _id(x):
    return np.asarray(x, dtype=np.float64)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    out, k = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[k:k + n].reshape(shape)
        k += n
    return out


def features(X):
    """Normalised inputs of raw (q, gamma, log R/theta_E, vphi), float32 as in the kernels."""
    X = np.asarray(X, dtype=np.float32)
    f = np.empty_like(X)
    f[:, 0] = (X[:, 0] - np.float32(0.75)) * np.float32(4.0)
    f[:, 1] = (X[:, 1] - np.float32(2.0)) * np.float32(1.0 / 0.3)
    f[:, 2] = X[:, 2] * np.float32(1.0 / 2.3)
    f[:, 3] = (X[:, 3] - np.float32(np.pi)) * np.float32(1.0 / np.pi)
    return f.astype(np.float64)


def sig(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(params, X, rounding=True):
    """Network output y [N, 2] and the cache of the backward pass.
    rounding=False: exact FP64 arithmetic (no BF16 rounding anywhere)."""
    bf16r = bf16 if rounding else _id
    P = unpack(params)
    a = bf16r(features(X))
    cache = [a]
    sps = []
    for l in range(1, 5):
        z = a @ bf16r(P[f"W{l}"]).T + P[f"b{l}"]
        s = sig(z)
        sps.append(bf16r(s * (1 + z * (1 - s))))
        a = bf16r(z * s)
        cache.append(a)
    y = a @ bf16r(P["W5"]).T + P["b5"]
    return y, (cache, sps, P)


def loss_grad(params, X, T, rounding=True):
    """Mean over rows of sum_o (y_o - T_o)^2 and its parameter gradient."""
    bf16 = globals()["bf16"] if rounding else _id
    y, (cache, sps, P) = forward(params, X, rounding)
    N = y.shape[0]
    e = y - T
    loss = float((e ** 2).sum() / N)
    g = {}
    dz = 2.0 * e / N
    g["b5"] = dz.sum(0)
    g["W5"] = bf16(dz).T @ cache[4]
    dA = bf16(dz) @ bf16(P["W5"])
    for l in range(4, 0, -1):
        dz = dA * sps[l - 1]
        g[f"b{l}"] = dz.sum(0)
        g[f"W{l}"] = bf16(dz).T @ cache[l - 1]
        if l > 1:
            dA = bf16(dz) @ bf16(P[f"W{l}"])
    flat = np.concatenate([g[name].ravel() for name, _ in SIZES])
    return loss, flat


def base_F(X):
    """1 + c1 z + c2 z^2 for raw inputs (q, gamma, ., vphi)."""
    X = np.asarray(X, dtype=np.float64)
    q, t, vp = X[:, 0], X[:, 1] - 1.0, X[:, 3]
    f = (1 - q) / (1 + q)
    z = -f * np.exp(2j * vp)
    c1 = t / (4 - t)
    c2 = c1 * (2 + t) / (6 - t)
    return 1 + c1 * z + c2 * z * z


def surrogate_F(params, X):
    """F predicted by the network: base terms + z^3 y / OUT_SCALE (complex),
    z = -f e^{2 i vphi}: the network stands for the series beyond its first
    two terms with the factor z^3 taken out."""
    y, _ = forward(params, X)
    X = np.asarray(X, dtype=np.float64)
    f = (1 - X[:, 0]) / (1 + X[:, 0])
    z = -f * np.exp(2j * X[:, 3])
    return base_F(X) + z ** 3 * (y[:, 0] + 1j * y[:, 1]) / OUT_SCALE
