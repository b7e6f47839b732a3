"""Pins of the learned-propagator oracle (oracle/nn.py): the circular 3x3
convolution against an FFT circular convolution, gradients against central
finite differences, GELU against its definition, bf16 rounding against
torch's bfloat16.  CPU only."""
import math

import numpy as np
import pytest

from oracle import nn


def test_conv3x3_matches_fft_circular_convolution():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 1, 7, 9))
    w = rng.standard_normal((1, 1, 3, 3))
    y = nn.conv3x3(x, w, np.zeros(1))
    K = np.zeros((7, 9))
    for di in range(3):
        for dj in range(3):
            K[(1 - di) % 7, (1 - dj) % 9] = w[0, 0, di, dj]
    want = np.real(np.fft.ifft2(np.fft.fft2(x[:, 0]) * np.fft.fft2(K)[None]))
    np.testing.assert_allclose(y[:, 0], want, rtol=1e-12, atol=1e-12)


def test_gelu_definition():
    z = np.linspace(-5, 5, 101)
    want = np.array([0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in z])
    np.testing.assert_allclose(nn.gelu(z), want, rtol=1e-14, atol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(nn.gelu_grad(z), (nn.gelu(z + h) - nn.gelu(z - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    ch = (1, 3, 2, 1)
    params = nn.init_params(3, ch)
    params = [(w * 3.0, rng.standard_normal(b.shape) * 0.1) for (w, b) in params]
    u = rng.standard_normal((2, 5, 6))
    target = rng.standard_normal((2, 5, 6))
    loss, grads = nn.loss_and_grads(params, u, target)
    h = 1e-6
    for li, (w, b) in enumerate(params):
        for idx in [(0, 0, 0, 0), (0, 0, 1, 2), (w.shape[0] - 1, w.shape[1] - 1, 2, 1)]:
            wp = w.copy(); wp[idx] += h
            wm = w.copy(); wm[idx] -= h
            pp = list(params); pp[li] = (wp, b)
            pm = list(params); pm[li] = (wm, b)
            fd = (nn.loss_and_grads(pp, u, target)[0] - nn.loss_and_grads(pm, u, target)[0]) / (2 * h)
            assert abs(fd - grads[li][0][idx]) <= 1e-6 * max(1.0, abs(fd)), (li, idx, fd, grads[li][0][idx])
        bp = b.copy(); bp[0] += h
        bm = b.copy(); bm[0] -= h
        pp = list(params); pp[li] = (w, bp)
        pm = list(params); pm[li] = (w, bm)
        fd = (nn.loss_and_grads(pp, u, target)[0] - nn.loss_and_grads(pm, u, target)[0]) / (2 * h)
        assert abs(fd - grads[li][1][0]) <= 1e-6 * max(1.0, abs(fd))


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(2).standard_normal(1000) * 10.0 ** np.random.default_rng(3).integers(-8, 8, 1000)
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(nn.bf16_round(x), want)
