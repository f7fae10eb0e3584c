"""FP64 reference of the two networks of Sec. 4 (classifier, initializer).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Architecture (the form the GPU kernels implement): inputs are the
standardised features u = (v - mean) / std of v = (z_1..z_nc, P, T) (the
scaling layer of Sec. 4.1.1), rounded to bfloat16; three hidden layers
a_l = bf16(silu(W_l a_{l-1} + b_l)) (Sec. 4.1.1: SiLU); a linear output
layer.  Weights are bfloat16, biases float32, sums exact here (FP64).
Parameters are one flat vector in the order W1, b1, W2, b2, W3, b3, W4, b4,
each W row-major [out, in].

Losses: classifier -- binary cross-entropy on the logit (Sec. 4.1.1,
Eq. bce with y = 1 stable), mean over the batch; initializer -- mean
absolute error of ln K summed over components (Sec. 4.2.1, Eq. mae), mean
over the batch.
"""
from __future__ import annotations

import numpy as np


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(a32)
    out[nan] = np.nan
    return out


def layer_sizes(din: int, hidden: int, dout: int):
    return [(hidden, din), (hidden, hidden), (hidden, hidden), (dout, hidden)]


def n_params(din: int, hidden: int, dout: int) -> int:
    return sum(o * i + o for o, i in layer_sizes(din, hidden, dout))


def unpack(theta, din, hidden, dout):
    Ws, bs, k = [], [], 0
    for o, i in layer_sizes(din, hidden, dout):
        Ws.append(np.asarray(theta[k:k + o * i], dtype=np.float64).reshape(o, i))
        k += o * i
        bs.append(np.asarray(theta[k:k + o], dtype=np.float64))
        k += o
    return Ws, bs


def silu(x):
    return x / (1.0 + np.exp(-x))


def dsilu(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def forward(theta, u, din, hidden, dout):
    """u: standardised inputs [n, din].  Returns outputs [n, dout] and the
    cache for backward.  Weights are used as bf16, as the kernels do."""
    Ws, bs = unpack(theta, din, hidden, dout)
    Ws = [bf16(W) for W in Ws]
    a = bf16(u)
    acts, pres = [a], []
    for l in range(3):
        pre = a @ Ws[l].T + bs[l]
        pres.append(pre)
        a = bf16(silu(pre))
        acts.append(a)
    out = a @ Ws[3].T + bs[3]
    return out, (Ws, acts, pres)


def loss_and_grad(theta, u, target, din, hidden, dout, kind):
    """kind 'bce' (target = 1 stable / 0 unstable, dout = 1) or 'mae'."""
    out, (Ws, acts, pres) = forward(theta, u, din, hidden, dout)
    n = u.shape[0]
    if kind == "bce":
        z = out[:, 0]
        loss = np.mean(np.logaddexp(0.0, z) - target * z)
        dout_ = ((1.0 / (1.0 + np.exp(-z))) - target)[:, None] / n
    else:
        d = out - target
        loss = np.mean(np.sum(np.abs(d), axis=1))
        dout_ = np.sign(d) / n
    grads = [None] * 8
    g = dout_
    for l in (3, 2, 1, 0):
        grads[2 * l] = g.T @ acts[l]
        grads[2 * l + 1] = g.sum(axis=0)
        if l > 0:
            da = g @ Ws[l]
            g = da * dsilu(pres[l - 1])
    flat = np.concatenate([x.reshape(-1) for x in grads])
    return loss, flat


def init_params(din, hidden, dout, rng):
    """He-style uniform initialisation (the draws the tests pass to the GPU)."""
    parts = []
    for o, i in layer_sizes(din, hidden, dout):
        lim = np.sqrt(6.0 / (i + o))
        parts.append(rng.uniform(-lim, lim, o * i))
        parts.append(np.zeros(o))
    return np.concatenate(parts)
