"""CPU oracle of the learned coarse propagator -- TEST INFRASTRUCTURE ONLY.

Psi_NN(u) = u + N(u), N = five 3x3 convolutions with circular padding,
1 -> 32 -> 32 -> 32 -> 32 -> 1 channels, GELU after the first four
(GELU(x) = x Phi(x), Phi the standard normal CDF), bias on every layer.
The paper allows any coarse propagator that approximates m fine steps
(Sec. 2.1, last paragraph: coarsening in space or order are its examples);
this network is one such choice, trained on (u, Phi^m u) pairs by mean
squared error.  Plain numpy in float64; arrays are NCHW, weights
[c_out][c_in][3][3].
"""
from __future__ import annotations

import math

import numpy as np

try:
    from scipy.special import erf as _erf
except ImportError:  # pragma: no cover
    _erf = np.vectorize(math.erf)

CHANNELS = (1, 32, 32, 32, 32, 1)


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[n,o,i,j] = b[o] + sum_{c,di,dj} w[o,c,di,dj] x[n,c,(i+di-1)%H,(j+dj-1)%W]."""
    n, c, h, wd = x.shape
    o = w.shape[0]
    y = np.zeros((n, o, h, wd)) + b[None, :, None, None]
    for di in range(3):
        for dj in range(3):
            xs = np.roll(x, shift=(1 - di, 1 - dj), axis=(2, 3))   # xs[i,j] = x[i+di-1, j+dj-1]
            y += np.einsum("oc,nchw->nohw", w[:, :, di, dj], xs)
    return y


def conv3x3_backward(x, w, dy):
    """Gradients of conv3x3 with respect to x, w and b, given dy."""
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for di in range(3):
        for dj in range(3):
            xs = np.roll(x, shift=(1 - di, 1 - dj), axis=(2, 3))
            dw[:, :, di, dj] = np.einsum("nohw,nchw->oc", dy, xs)
            g = np.einsum("oc,nohw->nchw", w[:, :, di, dj], dy)
            dx += np.roll(g, shift=(di - 1, dj - 1), axis=(2, 3))
    db = dy.sum(axis=(0, 2, 3))
    return dx, dw, db


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def init_params(seed: int = 0, channels=CHANNELS):
    """Seeded initial parameters (the shared draw of atm_inputs.conv_net_init:
    He-style uniform, last layer scaled by 0.1 so that Psi_NN starts near the
    identity)."""
    import atm_inputs as I
    return I.conv_net_init(seed, channels)


def forward(params, u):
    """u: (n, H, W).  Returns Psi_NN(u) and the cache for backward."""
    x = u[:, None]
    hs, zs = [x], []
    h = x
    for li, (w, b) in enumerate(params):
        z = conv3x3(h, w, b)
        zs.append(z)
        h = gelu(z) if li < len(params) - 1 else z
        hs.append(h)
    out = u + h[:, 0]
    return out, (hs, zs)


def loss_and_grads(params, u, target):
    """MSE = mean((Psi_NN(u) - target)^2) and its parameter gradients."""
    out, (hs, zs) = forward(params, u)
    diff = out - target
    loss = float(np.mean(diff * diff))
    g = (2.0 / diff.size) * diff[:, None]
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        w, b = params[li]
        dz = g if li == len(params) - 1 else g * gelu_grad(zs[li])
        dx, dw, db = conv3x3_backward(hs[li], w, dz)
        grads[li] = (dw, db)
        g = dx
    return loss, grads


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float64 values to bfloat16 (round to nearest even on the float32
    bit pattern) and back to float64."""
    f = np.asarray(a, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    bits = (bits + 0x7FFF + lsb) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)
