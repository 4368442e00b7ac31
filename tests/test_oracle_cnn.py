"""Pins of the network oracle: the circular convolution against a brute-force quadruple loop,
GELU against x * Phi(x) from scipy's normal distribution, and every parameter gradient
against central finite differences of the FP64 loss on a tiny net."""
import numpy as np
from scipy.stats import norm

from oracle import cnn


def test_conv_matches_brute_force():
    rng = np.random.default_rng(0)
    B, Ci, Co, N = 2, 3, 4, 5
    a = rng.standard_normal((B, Ci, N, N))
    W = rng.standard_normal((Co, Ci, 3, 3))
    b = rng.standard_normal(Co)
    got = cnn.conv(a, W, b)
    want = np.zeros_like(got)
    for bb in range(B):
        for co in range(Co):
            for y in range(N):
                for x in range(N):
                    s = b[co]
                    for ci in range(Ci):
                        for ky in range(3):
                            for kx in range(3):
                                s += W[co, ci, ky, kx] * a[bb, ci, (y + ky - 1) % N, (x + kx - 1) % N]
                    want[bb, co, y, x] = s
    assert np.allclose(got, want, atol=1e-12)


def test_gelu_definition():
    z = np.linspace(-6, 6, 1001)
    assert np.allclose(cnn.gelu(z), z * norm.cdf(z), atol=1e-14)
    h = 1e-6
    assert np.allclose(cnn.gelu_grad(z), (cnn.gelu(z + h) - cnn.gelu(z - h)) / (2 * h), atol=1e-8)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    dims = dict(in_ch=2, hidden=3, n_hidden=2, out_ch=2)
    cin, cout = cnn.layer_shapes(**dims)
    n = sum(co * ci * 9 + co for ci, co in zip(cin, cout))
    p = rng.standard_normal(n) * 0.4
    x = rng.standard_normal((2, 2, 5, 5))
    t = rng.standard_normal((2, 2, 5, 5))
    loss, g, _ = cnn.loss_and_grads(p, x, t, **dims)
    h = 1e-6
    fd = np.zeros(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd[i] = (cnn.loss_and_grads(p + e, x, t, **dims)[0] - cnn.loss_and_grads(p - e, x, t, **dims)[0]) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-9)
