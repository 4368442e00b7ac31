"""FP64 CPU oracle of the learned-initial-guess network (test infrastructure only).

The network is not from the paper; it is the small convolutional predictor of each time
step's initial guess.  conv3x3 with periodic (circular) padding,
  z[b, co, y, x] = bias[co] + sum_ci sum_{ky,kx} W[co, ci, ky, kx] a[b, ci, y+ky-1, x+kx-1],
GELU(z) = z Phi(z) with Phi the standard normal distribution function, mean-squared-error
loss; the backward pass is the chain rule written out layer by layer.  Parameters are one
flat vector, per layer W[cout][cin][3][3] then b[cout].
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def layer_shapes(in_ch, hidden, n_hidden, out_ch):
    L = n_hidden + 1
    cin = [in_ch] + [hidden] * (L - 1)
    cout = [hidden] * (L - 1) + [out_ch]
    return cin, cout


def unpack(params, in_ch, hidden, n_hidden, out_ch):
    cin, cout = layer_shapes(in_ch, hidden, n_hidden, out_ch)
    out, off = [], 0
    for ci, co in zip(cin, cout):
        W = params[off:off + co * ci * 9].reshape(co, ci, 3, 3).astype(np.float64)
        off += co * ci * 9
        b = params[off:off + co].astype(np.float64)
        off += co
        out.append((W, b))
    assert off == params.size
    return out


def shift(a, ky, kx):
    """a[..., y + ky - 1, x + kx - 1] with periodic indices."""
    return np.roll(a, shift=(1 - ky, 1 - kx), axis=(-2, -1))


def conv(a, W, b):
    B, ci_n, N, _ = a.shape
    z = np.zeros((B, W.shape[0], N, N)) + b[None, :, None, None]
    for ci in range(ci_n):
        for ky in range(3):
            for kx in range(3):
                z += W[None, :, ci, ky, kx, None, None] * shift(a[:, ci], ky, kx)[:, None]
    return z


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(layers, x):
    a, cache = x.astype(np.float64), []
    for l, (W, b) in enumerate(layers):
        z = conv(a, W, b)
        cache.append((a, z))
        a = gelu(z) if l + 1 < len(layers) else z
    return a, cache


def mse(out, target):
    d = out - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(layers, cache, g_out):
    """Gradients of the loss w.r.t. every layer's (W, b), given dLoss/d(output)."""
    grads = [None] * len(layers)
    g = g_out
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        a, z = cache[l]
        gW = np.zeros_like(W)
        for ci in range(W.shape[1]):
            for ky in range(3):
                for kx in range(3):
                    gW[:, ci, ky, kx] = np.einsum("bcyx,byx->c", g, shift(a[:, ci], ky, kx))
        gb = g.sum(axis=(0, 2, 3))
        grads[l] = (gW, gb)
        if l == 0:
            break
        ga = np.zeros_like(a)
        for ci in range(W.shape[1]):
            for ky in range(3):
                for kx in range(3):
                    # d/d a[ci, y, x] of W[co, ci, ky, kx] a[ci, y' + ky - 1, x' + kx - 1]
                    ga[:, ci] += np.roll(np.einsum("c,bcyx->byx", W[:, ci, ky, kx], g),
                                         shift=(ky - 1, kx - 1), axis=(-2, -1))
        g = ga * gelu_grad(cache[l - 1][1])
    return grads


def flat(grads):
    return np.concatenate([np.concatenate([gW.ravel(), gb.ravel()]) for gW, gb in grads])


def loss_and_grads(params, x, target, in_ch, hidden, n_hidden, out_ch):
    layers = unpack(np.asarray(params, dtype=np.float64), in_ch, hidden, n_hidden, out_ch)
    out, cache = forward(layers, x)
    loss, g = mse(out, target)
    return loss, flat(backward(layers, cache, g)), out
