"""FP64 reference of the two networks of Sec. 4 (classifier, initializer).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Architecture (the form the GPU kernels implement): inputs are the
standardised features u = (v - mean) / std of v = (z_1..z_nc, P, T) (the
scaling layer of Sec. 4.1.1), rounded to bfloat16; three hidden layers
a_l = bf16(silu(W_l a_{l-1} + b_l)) (Sec. 4.1.1: SiLU); a linear output
layer.  Weights are bfloat16, biases float32, sums exact here (FP64).
Parameters are one flat vector in the order W1, b1, W2, b2, W3, b3, W4, b4,
each W row-major [out, in].

Second architecture (arch 1, the initializer of Sec. 4.2.1): h_0 =
bf16(silu(W_0 u + b_0)); three residual blocks h_k = bf16(h_{k-1} +
bf16(silu(W_2k bf16(silu(W_{2k-1} h_{k-1} + b)) + b))); output W_7 [u; h_3]
+ b_7 (the wide shortcut concatenates the inputs with the last block's
output).  Parameters W_0, b_0, ..., W_7, b_7.

Losses: classifier -- binary cross-entropy on the logit (Sec. 4.1.1,
Eq. bce with y = 1 stable), mean over the batch; initializer -- mean
absolute error of ln K summed over components (Sec. 4.2.1, Eq. mae), mean
over the batch; second stage of the initializer ('mae_theta', Sec. 4.2.2)
-- that plus w |theta - theta_hat|, theta_hat the Rachford-Rice root for
the predicted K, differentiated by the implicit-function theorem.
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


def layer_sizes(din: int, hidden: int, dout: int, arch: int = 0):
    if arch == 1:
        return [(hidden, din)] + [(hidden, hidden)] * 6 + [(dout, din + hidden)]
    return [(hidden, din), (hidden, hidden), (hidden, hidden), (dout, hidden)]


def n_params(din: int, hidden: int, dout: int, arch: int = 0) -> int:
    return sum(o * i + o for o, i in layer_sizes(din, hidden, dout, arch))


def unpack(theta, din, hidden, dout, arch=0):
    Ws, bs, k = [], [], 0
    for o, i in layer_sizes(din, hidden, dout, arch):
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


def forward(theta, u, din, hidden, dout, arch=0):
    """u: standardised inputs [n, din].  Returns outputs [n, dout] and the
    cache for backward.  Weights are used as bf16, as the kernels do."""
    Ws, bs = unpack(theta, din, hidden, dout, arch)
    Ws = [bf16(W) for W in Ws]
    a = bf16(u)
    if arch == 1:
        pres, acts = [], [a]
        pre = a @ Ws[0].T + bs[0]
        pres.append(pre)
        h = bf16(silu(pre))
        hs = [h]
        for k in range(1, 4):
            pa = h @ Ws[2 * k - 1].T + bs[2 * k - 1]
            ak = bf16(silu(pa))
            pc = ak @ Ws[2 * k].T + bs[2 * k]
            ck = bf16(silu(pc))
            pres += [pa, pc]
            acts.append(ak)
            h = bf16(h + ck)
            hs.append(h)
        out = np.concatenate([a, h], axis=1) @ Ws[7].T + bs[7]
        return out, (Ws, acts, pres, hs)
    acts, pres = [a], []
    for l in range(3):
        pre = a @ Ws[l].T + bs[l]
        pres.append(pre)
        a = bf16(silu(pre))
        acts.append(a)
    out = a @ Ws[3].T + bs[3]
    return out, (Ws, acts, pres)


def rr_theta(z, lnK):
    """Rachford-Rice root (Eq. RR) for one mixture by bisection on the
    Leibovici-Neoschil window (Appendix C) and d theta / d ln K from the
    implicit-function theorem (Sec. 4.2.2): d theta / d K_i = -f_K_i / f_theta.
    None if K does not bracket 1."""
    K = np.exp(lnK)
    if not (K.max() > 1.0 and K.min() < 1.0):
        return None
    lo, hi = 1.0 / (1.0 - K.max()), 1.0 / (1.0 - K.min())
    f = lambda t: np.sum(z * (K - 1.0) / (1.0 + (K - 1.0) * t))
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0.0:
            lo = mid
        else:
            hi = mid
    th = 0.5 * (lo + hi)
    t = 1.0 + (K - 1.0) * th
    f_K = z / t ** 2                                   # d f / d K_i
    f_th = -np.sum(z * (K - 1.0) ** 2 / t ** 2)        # d f / d theta
    return th, -(f_K / f_th) * K                       # d theta / d ln K_i


def loss_and_grad(theta, u, target, din, hidden, dout, kind, arch=0, wth=0.0, z=None, th_target=None):
    """kind 'bce' (target = 1 stable / 0 unstable, dout = 1), 'mae', or
    'mae_theta' (also z [n, dout] and th_target [n]; weight wth)."""
    cache = forward(theta, u, din, hidden, dout, arch)
    out = cache[0]
    n = u.shape[0]
    if kind == "bce":
        zz = out[:, 0]
        loss = np.mean(np.logaddexp(0.0, zz) - target * zz)
        g = ((1.0 / (1.0 + np.exp(-zz))) - target)[:, None] / n
    else:
        d = out - target
        loss = np.mean(np.sum(np.abs(d), axis=1))
        g = np.sign(d) / n
        if kind == "mae_theta":
            for m in range(n):
                r = rr_theta(z[m], out[m])
                if r is None:
                    continue
                th, dth = r
                e = th - th_target[m]
                loss += wth * abs(e) / n
                g[m] += wth * np.sign(e) * dth / n
    return loss, backward(cache, g, din, hidden, dout, arch)


def backward(cache, g, din, hidden, dout, arch=0):
    """Gradient of the parameters given d loss / d output g [n, dout]."""
    if arch == 1:
        out, (Ws, acts, pres, hs) = cache
        grads = [None] * 16
        inp = np.concatenate([acts[0], hs[3]], axis=1)
        grads[14] = g.T @ inp
        grads[15] = g.sum(axis=0)
        dh = (g @ Ws[7])[:, din:]
        for k in (3, 2, 1):
            dpc = dh * dsilu(pres[2 * k])
            grads[4 * k] = dpc.T @ acts[k]
            grads[4 * k + 1] = dpc.sum(axis=0)
            dpa = (dpc @ Ws[2 * k]) * dsilu(pres[2 * k - 1])
            grads[4 * k - 2] = dpa.T @ hs[k - 1]
            grads[4 * k - 1] = dpa.sum(axis=0)
            dh = dh + dpa @ Ws[2 * k - 1]
        dp0 = dh * dsilu(pres[0])
        grads[0] = dp0.T @ acts[0]
        grads[1] = dp0.sum(axis=0)
        return np.concatenate([x.reshape(-1) for x in grads])
    out, (Ws, acts, pres) = cache
    grads = [None] * 8
    for l in (3, 2, 1, 0):
        grads[2 * l] = g.T @ acts[l]
        grads[2 * l + 1] = g.sum(axis=0)
        if l > 0:
            da = g @ Ws[l]
            g = da * dsilu(pres[l - 1])
    return np.concatenate([x.reshape(-1) for x in grads])


def init_params(din, hidden, dout, rng, arch=0):
    """Glorot-uniform initialisation (the draws the tests pass to the GPU)."""
    parts = []
    for o, i in layer_sizes(din, hidden, dout, arch):
        lim = np.sqrt(6.0 / (i + o))
        parts.append(rng.uniform(-lim, lim, o * i))
        parts.append(np.zeros(o))
    return np.concatenate(parts)
