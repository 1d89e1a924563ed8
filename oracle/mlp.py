"""FP64 reference of the troubled-cell gate network (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use this
module; it shares no code with the CUDA path.

The gate is not part of the paper. It predicts, per cell, whether the
nonlinear WENO weights of the compact reconstruction (Sec. 3.4) depart from
the linear ones, from 24 inputs (the cell and its three face neighbours, for
eta1 and h2: deviation of the average from the four-cell mean and the
size-scaled gradient, normalised). The network is

    s = w3 . relu(W2 relu(W1 x' + b1) + b2) + b3,   x' = (x - mean) * inv_std,

24 -> 32 -> 32 -> 1, trained on the weighted logistic loss

    L = sum_i pos_w y_i softplus(-s_i) + (1 - y_i) softplus(s_i).

The parameter vector is W1[32][24], b1[32], W2[32][32], b2[32], w3[32], b3,
mean[24], inv_std[24]; the first NTRAIN entries are trained.

With `use_bf16=True` the operands of the products are rounded to bfloat16
(round to nearest, ties to even) where a BF16 tensor-core implementation
with FP32 sums rounds them, in two conventions:
- inference (`forward`): the normalisation is folded into the first layer,
  W1' = W1 diag(inv_std), b1' = b1 - W1' mean; the raw inputs, W1', W2 and
  both hidden activations are rounded;
- training (`loss_grad`): the normalised inputs, W1, W2, both hidden
  activations and the output gradients dZ2, dZ1 that enter the
  weight-gradient and back-propagation products are rounded.
In exact arithmetic both are the network above. Everything else is FP64.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 24, 32
W1, B1 = 0, N_H * N_IN
W2 = B1 + N_H
B2 = W2 + N_H * N_H
W3 = B2 + N_H
B3 = W3 + N_H
MEAN = B3 + 1
ISTD = MEAN + N_IN
NPARAM = ISTD + N_IN
NTRAIN = MEAN


def unpack(P):
    P = np.asarray(P, dtype=np.float64)
    assert P.shape == (NPARAM,)
    return dict(W1=P[W1:B1].reshape(N_H, N_IN), b1=P[B1:W2], W2=P[W2:B2].reshape(N_H, N_H), b2=P[B2:W3],
                w3=P[W3:B3], b3=P[B3], mean=P[MEAN:ISTD], istd=P[ISTD:NPARAM])


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), via float32, as float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def _normalise(p, X, use_bf16):
    if use_bf16:
        # the kernels form (x - mean) * inv_std in FP32, then round
        x32 = (np.asarray(X, np.float32) - p["mean"].astype(np.float32)) * p["istd"].astype(np.float32)
        return bf16(x32)
    return (np.asarray(X, np.float64) - p["mean"]) * p["istd"]


def forward(P, X, use_bf16=False):
    """Logits s[n] of samples X[n][24] (inference convention)."""
    if not use_bf16:
        return _forward(P, X, False)[0]
    p = unpack(P)
    w1 = bf16((p["W1"].astype(np.float32) * p["istd"].astype(np.float32)[None, :]).astype(np.float64))
    b1 = p["b1"] - (p["W1"] * p["istd"][None, :]) @ p["mean"]
    x = bf16(np.asarray(X, np.float32))
    h1 = bf16(np.maximum(x @ w1.T + b1, 0.0))
    h2 = bf16(np.maximum(h1 @ bf16(p["W2"]).T + p["b2"], 0.0))
    return h2 @ p["w3"] + p["b3"]


def _forward(P, X, use_bf16):
    """Logits and intermediate values (training convention)."""
    p = unpack(P)
    r = bf16 if use_bf16 else (lambda a: np.asarray(a, np.float64))
    x = _normalise(p, X, use_bf16)
    w1, w2 = r(p["W1"]), r(p["W2"])
    z1 = x @ w1.T + p["b1"]
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ w2.T + p["b2"]
    h2 = r(np.maximum(z2, 0.0))
    s = h2 @ p["w3"] + p["b3"]
    return s, dict(x=x, w1=w1, w2=w2, z1=z1, h1=h1, z2=z2, h2=h2, p=p)


def softplus(s):
    return np.maximum(s, 0.0) + np.log1p(np.exp(-np.abs(s)))


def sigmoid(s):
    return 0.5 * (1.0 + np.tanh(0.5 * s))


def loss(P, X, y, pos_w, use_bf16=False):
    s, _ = _forward(P, X, use_bf16)
    y = np.asarray(y, np.float64)
    return float(np.sum(pos_w * y * softplus(-s) + (1 - y) * softplus(s)))


def loss_grad(P, X, y, pos_w, use_bf16=False):
    """Loss and its gradient (NTRAIN entries, summed over the samples)."""
    r = bf16 if use_bf16 else (lambda a: np.asarray(a, np.float64))
    s, c = _forward(P, X, use_bf16)
    p = c["p"]
    y = np.asarray(y, np.float64)
    L = float(np.sum(pos_w * y * softplus(-s) + (1 - y) * softplus(s)))
    ds = -pos_w * y * sigmoid(-s) + (1 - y) * sigmoid(s)          # dL/ds
    g = np.zeros(NTRAIN)
    g[W3:B3] = c["h2"].T @ ds
    g[B3] = ds.sum()
    dz2 = ds[:, None] * p["w3"][None, :] * (c["z2"] > 0)         # dL/dz2
    g[B2:W3] = dz2.sum(0)
    g[W2:B2] = (r(dz2).T @ c["h1"]).ravel()
    dz1 = (r(dz2) @ c["w2"]) * (c["z1"] > 0)                       # dL/dz1
    g[B1:W2] = dz1.sum(0)
    g[W1:B1] = (r(dz1).T @ c["x"]).ravel()
    return L, g


def adam(P, G, m, v, step, lr, scale, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba) on the first NTRAIN parameters, in place."""
    gr = G * scale
    m[:] = b1 * m + (1 - b1) * gr
    v[:] = b2 * v + (1 - b2) * gr * gr
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    P[:NTRAIN] -= lr * mh / (np.sqrt(vh) + eps)
