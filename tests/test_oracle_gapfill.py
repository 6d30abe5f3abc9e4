"""Pins for the gap-filling oracle (constrained Gaussian realisation with a symmetric band
covariance): the dense conditional mean and the special cases that fix it."""
import numpy as np
import pytest
from scipy.linalg import toeplitz

import oracle
import synth
from oracle import gapfill as og


def dense_band(taps, ns):
    col = np.zeros(ns)
    k = min(len(taps), ns)
    col[:k] = taps[:k]
    return toeplitz(col)


@pytest.fixture(scope="module")
def case():
    oracle.build()
    g = np.random.default_rng(11)
    ns, nd = 400, 3
    taps = np.stack([synth.noise_covariance_band(64) * s for s in (1.0, 0.5, 2.0)])
    n = synth.band_realization(taps, ns, g)
    d = synth.band_realization(taps, ns, g) + 3.0
    valid = g.random((nd, ns)) > 0.15
    valid[:, 120:170] = False      # a long gap
    valid[1, :5] = False           # a gap at the start of a stream
    return taps, d, n, valid


def test_matches_the_dense_conditional_mean(case):
    taps, d, n, valid = case
    out, it = og.gapfill(taps, d, valid, n, tol=1e-13)
    for i in range(d.shape[0]):
        N = dense_band(taps[i], d.shape[1])
        v, gmask = valid[i], ~valid[i]
        ref = n[i, gmask] + N[np.ix_(gmask, v)] @ np.linalg.solve(N[np.ix_(v, v)], d[i, v] - n[i, v])
        assert np.allclose(out[i, gmask], ref, rtol=0, atol=1e-9 * np.abs(ref).max())
        assert np.array_equal(out[i, v], d[i, v])


def test_special_cases(case):
    taps, d, n, valid = case
    out, _ = og.gapfill(taps, d, np.ones_like(valid), n)
    assert np.array_equal(out, d)                       # nothing to fill
    out, it = og.gapfill(taps, d, np.zeros_like(valid), n)
    assert np.array_equal(out, n) and np.all(it == 0)   # nothing observed: the realisation itself
    out, it = og.gapfill(taps, n, valid, n)
    assert np.array_equal(out, n) and np.all(it == 0)   # data equal to the realisation
    white = taps[:, :1]
    out, _ = og.gapfill(white, d, valid, n)
    assert np.allclose(out, np.where(valid, d, n), rtol=0, atol=1e-12)   # no correlation to borrow


def test_covariance_band_is_positive_definite():
    for k in (16, 64, 1024):
        c = synth.noise_covariance_band(k)
        w = np.linspace(0, np.pi, 1 << 14)
        assert (c[0] + 2 * np.cos(np.outer(w, np.arange(1, k))) @ c[1:]).min() > 0
