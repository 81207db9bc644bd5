"""Oracle: FP64 multilayer perceptron forward/backward with optional BF16 rounding emulation.

TEST INFRASTRUCTURE ONLY.  The network follows the surrogate of the chemistry step: a plain
stack of dense layers with GELU activations (§2 states GELU activations and Adam training for
the paper's per-species networks); here the layers are x -> 512 -> 512 -> 512 -> 512 -> out.

Conventions: W[l] has shape [n_out, n_in]; y = x @ W.T + b.  GELU is the exact form
x * Phi(x) = 0.5 x (1 + erf(x / sqrt 2)).  BF16 emulation rounds a value first to FP32 and then
to BF16 with round-to-nearest-even, at the points where the GPU path holds BF16 data: the
weights of layers 2-5 and each hidden activation after GELU.  The first layer is compensated:
the input x and the weights W each become a pair of BF16 numbers, hi = bf16(v) and
lo = bf16(v - hi), and the layer computes x_hi W_hi^T + x_lo W_hi^T + x_hi W_lo^T (the lo*lo
product is left out).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def bf16_round(x):
    """Round to the nearest BF16 value (ties to even), via FP32.  Returns float64."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    bias = ((u >> 16) & 1) + 0x7FFF
    r = ((u + bias) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    # NaN / Inf pass through unchanged
    bad = ~np.isfinite(f)
    if np.any(bad):
        out = np.where(bad, f.astype(np.float64), out)
    return out


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def split_bf16(v):
    """(hi, lo): hi = bf16(v), lo = bf16(v - hi).  hi + lo carries about 16 significant bits."""
    v = np.asarray(v, np.float64)
    hi = bf16_round(v)
    return hi, bf16_round(v - hi)


def first_layer(W, x):
    """Compensated BF16 product x W^T of the first layer (no bias)."""
    xh, xl = split_bf16(x)
    wh, wl = split_bf16(W)
    return xh @ wh.T + xl @ wh.T + xh @ wl.T


def forward(Ws, bs, x, emulate_bf16=True):
    """Returns (output [M, n_out], cache).  cache holds the layer inputs a[l] and pre-activations z[l]."""
    rnd = bf16_round if emulate_bf16 else (lambda v: np.asarray(v, np.float64))
    if emulate_bf16:
        xh, xl = split_bf16(x)
        a = xh + xl                # the input the first layer's weight gradient sees
    else:
        a = np.asarray(x, np.float64)
    acts, pres = [a], []
    L = len(Ws)
    for l in range(L):
        if l == 0 and emulate_bf16:
            z = first_layer(Ws[0], x) + np.asarray(bs[0], np.float64)
            pres.append(z)
            a = rnd(gelu(z)) if L > 1 else z
            if L > 1:
                acts.append(a)
            continue
        W = rnd(Ws[l])
        z = a @ W.T + np.asarray(bs[l], np.float64)
        pres.append(z)
        if l < L - 1:
            a = rnd(gelu(z))
            acts.append(a)
        else:
            a = z
    return a, {"a": acts, "z": pres}


def mse_loss(out, target):
    d = out - target
    return float(np.mean(d * d))


def backward(Ws, bs, cache, out, target, emulate_bf16=False):
    """Gradients of mean((out - target)^2) with respect to every W[l] and b[l] (FP64)."""
    rnd = bf16_round if emulate_bf16 else (lambda v: np.asarray(v, np.float64))
    M = out.shape[0]
    n_out = out.shape[1]
    dz = 2.0 * (out - target) / (M * n_out)
    L = len(Ws)
    dW = [None] * L
    db = [None] * L
    for l in range(L - 1, -1, -1):
        a_in = cache["a"][l]
        dW[l] = dz.T @ a_in
        db[l] = dz.sum(axis=0)
        if l > 0:
            da = dz @ rnd(Ws[l])
            dz = da * gelu_grad(cache["z"][l - 1])
    return dW, db


def adam_step(params, grads, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction, in place on FP64 arrays."""
    for i in range(len(params)):
        m[i] = beta1 * m[i] + (1.0 - beta1) * grads[i]
        v[i] = beta2 * v[i] + (1.0 - beta2) * grads[i] * grads[i]
        mh = m[i] / (1.0 - beta1 ** step)
        vh = v[i] / (1.0 - beta2 ** step)
        params[i] = params[i] - lr * mh / (np.sqrt(vh) + eps)
    return params, m, v
