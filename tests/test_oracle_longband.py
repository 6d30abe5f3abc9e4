"""Pins for the oracle's symmetric band N^-1 at the long lengths of the overlap-save evaluation
(SymmetricBandToeplitzOperator, Table 2): the oracle keeps the direct sum, checked here against
dense Toeplitz matrices and numpy FFTs."""
import numpy as np
import pytest
import scipy.linalg

import synth


@pytest.mark.parametrize("ntaps,ns", [(65, 64), (300, 100), (300, 1000), (1024, 700), (2048, 3000)])
def test_long_band_matches_dense_toeplitz(orc, ntaps, ns):
    taps = synth.inverse_noise_taps(ntaps)
    x = np.random.default_rng(ntaps + ns).normal(size=(2, ns))
    col = np.zeros(ns)
    k = min(ns, ntaps)
    col[:k] = taps[:k]
    T = scipy.linalg.toeplitz(col)
    y = orc.ninv_band(np.stack([taps, 0.5 * taps]), x)
    np.testing.assert_allclose(y[0], T @ x[0], rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(y[1], 0.5 * (T @ x[1]), rtol=1e-11, atol=1e-14)


def test_long_band_matches_fft_circular_convolution_interior(orc):
    ntaps, ns = 2048, 1 << 14
    taps = synth.inverse_noise_taps(ntaps)
    x = np.random.default_rng(5).normal(size=(1, ns))
    kern = np.zeros(ns)
    kern[:ntaps] = taps
    kern[-(ntaps - 1):] = taps[1:][::-1]
    ycirc = np.fft.irfft(np.fft.rfft(x[0]) * np.fft.rfft(kern), n=ns)
    y = orc.ninv_band(taps, x)[0]
    h = ntaps - 1
    np.testing.assert_allclose(y[h:ns - h], ycirc[h:ns - h], rtol=1e-10, atol=1e-12 * np.abs(ycirc).max())


@pytest.mark.parametrize("ntaps", [256, 2048])
def test_long_band_symmetric_and_positive_definite(orc, ntaps):
    taps = synth.inverse_noise_taps(ntaps)
    g = np.random.default_rng(6)
    x, y = g.normal(size=(2, 1, 5000))
    a = np.dot(x[0], orc.ninv_band(taps, y)[0])
    b = np.dot(orc.ninv_band(taps, x)[0], y[0])
    assert abs(a - b) < 1e-12 * abs(a)
    w = np.linspace(0, np.pi, 1 << 15)
    symbol = taps[0] + 2 * np.cos(np.outer(w, np.arange(1, ntaps))) @ taps[1:]
    assert symbol.min() > 0
