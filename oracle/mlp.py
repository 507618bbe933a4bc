"""FP64 reference of the duration surrogate -- TEST INFRASTRUCTURE ONLY.

The surrogate is the project's own addition (the paper has no learned
component): an MLP 28 -> 256 -> 256 -> 256 -> 2 with ReLU that predicts
(log T*, feasibility logit) of an edge from its boundary states.  Its
precision scheme is part of its definition and is reproduced here exactly:

  forward   x_b = bf16(x);  z_l = h_{l-1,b} W_l,b + b_l;  h_l = relu(z_l);
            h_l,b = bf16(h_l)  (l = 1..3);  y = h_3,b W_4,b + b_4
  loss      L = (1/n) sum_i [ f_i (y_i0 - log T*_i)^2 + BCE(y_i1, f_i) ]
  backward  dz_4 = dL/dy;  dW_l = h_{l-1,b}^T bf16(dz_l);  db_l = sum_i dz_l;
            dz_{l-1} = (bf16(dz_l) W_l,b^T) * 1[z_{l-1} > 0]
  Adam      on FP32 master weights; W_b = bf16(master)

with bf16() round-to-nearest-even.  Everything else is float64.
Features: q scaled by the joint box to [-1, 1], qd by qd_max, for both
states (28 values, zero-padded to 32).
"""
from __future__ import annotations

import numpy as np

DIMS = (32, 256, 256, 256, 2)   # input padded from 28 to 32


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(x, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(a)
    if np.any(nan):
        out = np.where(nan, np.nan, out)
    return out


def features(arm, s0, s1):
    lo = arm["q_lo"].astype(np.float64)
    hi = arm["q_hi"].astype(np.float64)
    c, h = 0.5 * (lo + hi), 0.5 * (hi - lo)
    vm = arm["qd_max"].astype(np.float64)
    s0 = np.asarray(s0, np.float64)
    s1 = np.asarray(s1, np.float64)
    X = np.zeros((s0.shape[0], 32))
    X[:, 0:7] = (s0[:, 0:7] - c) / h
    X[:, 7:14] = s0[:, 8:15] / vm
    X[:, 14:21] = (s1[:, 0:7] - c) / h
    X[:, 21:28] = s1[:, 8:15] / vm
    return X


def forward(params, X, rnd=bf16):
    """params: list of (W [in][out] float64 master, b [out]).  Returns y and
    the cache needed by backward.  `rnd` is the rounding of the stored
    operands (bf16; the identity gives the exact FP64 network)."""
    h = rnd(X)
    cache = [h]
    zs = []
    for l, (W, b) in enumerate(params):
        z = h @ rnd(W) + b
        zs.append(z)
        if l < len(params) - 1:
            h = rnd(np.maximum(z, 0.0))
            cache.append(h)
    return zs[-1], (cache, zs)


def loss_and_grad_y(y, logT, feas):
    n = y.shape[0]
    f = feas.astype(np.float64)
    d = y[:, 0] - np.where(feas, logT, 0.0)
    s = 1.0 / (1.0 + np.exp(-y[:, 1]))
    bce = np.maximum(y[:, 1], 0) - y[:, 1] * f + np.log1p(np.exp(-np.abs(y[:, 1])))
    L = np.sum(f * d * d + bce) / n
    dy = np.zeros_like(y)
    dy[:, 0] = 2.0 * f * d / n
    dy[:, 1] = (s - f) / n
    return L, dy


def backward(params, cache, dy, rnd=bf16):
    hs, zs = cache
    grads = [None] * len(params)
    dz = dy
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        dzb = rnd(dz)
        grads[l] = (hs[l].T @ dzb, dz.sum(axis=0))
        if l > 0:
            dh = dzb @ rnd(W).T
            dz = dh * (zs[l - 1] > 0)
    return grads


def adam(params, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step on float64 copies (t is the 1-based step count)."""
    out, m2, v2 = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        res = []
        for p, g, mm, vv in ((W, gW, mW, vW), (b, gb, mb, vb)):
            mm = b1 * mm + (1 - b1) * g
            vv = b2 * vv + (1 - b2) * g * g
            mh = mm / (1 - b1 ** t)
            vh = vv / (1 - b2 ** t)
            res.append((p - lr * mh / (np.sqrt(vh) + eps), mm, vv))
        out.append((res[0][0], res[1][0]))
        m2.append((res[0][1], res[1][1]))
        v2.append((res[0][2], res[1][2]))
    return out, m2, v2
