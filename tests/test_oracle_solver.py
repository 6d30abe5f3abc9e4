"""Pins for the oracle's solver: dense normal equations, one-step convergence, noiseless
recovery, monotone energy error, and finite-difference gradients of chi^2."""
import numpy as np
import pytest
import scipy.linalg

import synth


def _dense_P(npix, pix, c, s):
    """Dense pointing matrix [nsamp_total][3 npix] from per-sample pixel and weights."""
    n = pix.size
    A = np.zeros((n, 3 * npix))
    r = np.arange(n)
    p = pix.ravel()
    A[r, 3 * p] = 1.0
    A[r, 3 * p + 1] = c.ravel()
    A[r, 3 * p + 2] = s.ravel()
    return A


def _dense_band(taps, ns):
    col = np.zeros(ns)
    k = min(ns, taps.size)
    col[:k] = taps[:k]
    return scipy.linalg.toeplitz(col)


@pytest.fixture(scope="module")
def tiny(orc):
    """nside 1 (36 unknowns), 6 hex detectors x 3000 samples, banded noise."""
    obs = synth.Observation(1, synth.satellite_scan(3000), synth.hex_focal_plane(6))
    pix, c, s, _ = orc.pointing(obs.nside, obs.q_bore, obs.q_det)
    taps = np.tile(synth.inverse_noise_taps(), (6, 1))
    taps[1] *= 0.5
    return obs, pix, c, s, orc.Noise(taps=taps)


def test_dense_normal_equations(orc, tiny):
    obs, pix, c, s, noise = tiny
    nd, ns = pix.shape
    A = _dense_P(obs.npix, pix, c, s)
    Ninv = scipy.linalg.block_diag(*[_dense_band(noise.taps[j], ns) for j in range(nd)])
    ATA = A.T @ Ninv @ A
    g = np.random.default_rng(0)
    x = g.normal(size=(obs.npix, 3))
    d = g.normal(size=(nd, ns))
    np.testing.assert_allclose(orc.apply_ata(obs.npix, pix, c, s, noise, None, x).ravel(), ATA @ x.ravel(), rtol=1e-10, atol=1e-12)
    b = orc.rhs(obs.npix, pix, c, s, noise, None, d)
    np.testing.assert_allclose(b.ravel(), A.T @ Ninv @ d.ravel(), rtol=1e-10, atol=1e-12)
    bj = orc.bj(obs.npix, pix, c, s, noise)
    v = bj["valid"]
    assert v.sum() >= 4
    sel = np.repeat(v, 3)
    bv = orc.rhs(obs.npix, pix, c, s, noise, v, d)
    assert np.all(bv[~v] == 0)
    xs, it, hist = orc.pcg(obs.npix, pix, c, s, noise, v, bj["inv"], bv, maxiter=200, tol=1e-13)
    ref = np.linalg.solve(ATA[np.ix_(sel, sel)], bv.ravel()[sel])
    np.testing.assert_allclose(xs.ravel()[sel], ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
    assert np.all(xs[~v] == 0)
    assert hist[-1] <= 1e-13
    # masked operator S A S^T, applied to a vector that is not zero on the masked pixels
    S = np.diag(sel.astype(float))
    got = orc.apply_ata(obs.npix, pix, c, s, noise, v, x).ravel()
    np.testing.assert_allclose(got, S @ ATA @ S @ x.ravel(), rtol=1e-10, atol=1e-12)


def test_energy_error_decreases(orc, tiny):
    obs, pix, c, s, noise = tiny
    nd, ns = pix.shape
    A = _dense_P(obs.npix, pix, c, s)
    Ninv = scipy.linalg.block_diag(*[_dense_band(noise.taps[j], ns) for j in range(nd)])
    ATA = A.T @ Ninv @ A
    b = orc.rhs(obs.npix, pix, c, s, noise, None, np.random.default_rng(1).normal(size=(nd, ns)))
    bj = orc.bj(obs.npix, pix, c, s, noise)
    v = bj["valid"]
    sel = np.repeat(v, 3)
    b[~v] = 0
    Av = ATA[np.ix_(sel, sel)]
    ref = np.linalg.solve(Av, b.ravel()[sel])
    errs = []
    for k in range(1, 12):
        x, _, _ = orc.pcg(obs.npix, pix, c, s, noise, v, bj["inv"], b, maxiter=k, tol=0.0)
        e = x.ravel()[sel] - ref
        errs.append(e @ Av @ e)
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-9) for i in range(len(errs) - 1))


def test_white_noise_one_step_is_binned_map(orc):
    """White noise makes P^T N^-1 P exactly block diagonal, equal to the BJ blocks, so PCG
    with that preconditioner lands on the binned map after one step."""
    obs, sky, noise, sigma2 = synth.config1(nsamp=65536, nside=16)
    pix, c, s, _ = orc.pointing(obs.nside, obs.q_bore, obs.q_det)
    d = orc.P(pix, c, s, sky) + noise
    nz = orc.Noise(sigma2=sigma2)
    bj = orc.bj(obs.npix, pix, c, s, nz)
    b = orc.rhs(obs.npix, pix, c, s, nz, bj["valid"], d)
    binned = orc.binned_map(bj, b)
    x, it, hist = orc.pcg(obs.npix, pix, c, s, nz, bj["valid"], bj["inv"], b, maxiter=30, tol=1e-8)
    assert it == 1
    assert hist[1] < 1e-13
    v = bj["valid"]
    np.testing.assert_allclose(x[v], binned[v], rtol=1e-12, atol=1e-12 * np.abs(binned).max())


def test_noiseless_recovery_banded(orc):
    obs = synth.Observation(8, synth.satellite_scan(16384), synth.hex_focal_plane(12))
    pix, c, s, _ = orc.pointing(obs.nside, obs.q_bore, obs.q_det)
    taps = np.tile(synth.inverse_noise_taps(), (12, 1))
    nz = orc.Noise(taps=taps)
    bj = orc.bj(obs.npix, pix, c, s, nz)
    v = bj["valid"]
    m_true = synth.gaussian_sky(obs.nside, synth.rng(9, 0))
    m_true[~v] = 0.0
    d = orc.P(pix, c, s, m_true)
    b = orc.rhs(obs.npix, pix, c, s, nz, v, d)
    x, it, hist = orc.pcg(obs.npix, pix, c, s, nz, v, bj["inv"], b, maxiter=500, tol=1e-13)
    err = np.linalg.norm(x[v] - m_true[v]) / np.linalg.norm(m_true[v])
    assert err < 1e-10


def test_noiseless_recovery_white(orc):
    obs, sky, _, sigma2 = synth.config1(nsamp=65536, nside=16)
    pix, c, s, _ = orc.pointing(obs.nside, obs.q_bore, obs.q_det)
    nz = orc.Noise(sigma2=sigma2)
    bj = orc.bj(obs.npix, pix, c, s, nz)
    v = bj["valid"]
    sky[~v] = 0.0
    b = orc.rhs(obs.npix, pix, c, s, nz, v, orc.P(pix, c, s, sky))
    x, it, _ = orc.pcg(obs.npix, pix, c, s, nz, v, bj["inv"], b, maxiter=30, tol=1e-8)
    assert np.linalg.norm(x[v] - sky[v]) / np.linalg.norm(sky[v]) < 1e-12


def _chi2(orc, obs, delta, m, d, nz):
    pix, c, s, _ = orc.pointing(obs.nside, obs.q_bore, obs.q_det, psi_offset=delta)
    return orc.chi2_grad(obs.npix, pix, c, s, nz, m, d, want_grad=False)[0]


def test_gradients_match_central_differences(orc):
    """d chi^2/d delta_j and d chi^2/d m by central differences, h = 1e-6, FP64."""
    nd, ns = 8, 1 << 14
    obs = synth.Observation(16, synth.satellite_scan(ns), synth.hex_focal_plane(nd))
    g = synth.rng(5, 3)
    delta_true = np.radians(g.normal(0, 1.0, nd))
    sky = synth.gaussian_sky(obs.nside, g)
    taps = np.tile(synth.inverse_noise_taps(), (nd, 1))
    nz = orc.Noise(taps=taps)
    pix, c, s, _ = orc.pointing(obs.nside, obs.q_bore, obs.q_det, psi_offset=delta_true)
    d = orc.P(pix, c, s, sky) + synth.one_over_f_noise(nd, ns, g)
    delta = delta_true / 2
    m = sky * 1.01
    pix, c, s, _ = orc.pointing(obs.nside, obs.q_bore, obs.q_det, psi_offset=delta)
    chi2, gm, gp = orc.chi2_grad(obs.npix, pix, c, s, nz, m, d)
    h = 1e-6
    for j in range(nd):
        e = np.zeros(nd); e[j] = h
        fd = (_chi2(orc, obs, delta + e, m, d, nz) - _chi2(orc, obs, delta - e, m, d, nz)) / (2 * h)
        # FD error ~ eps chi2 / h + h^2 |chi2'''|; both far below 1e-5 relative of the scale
        assert abs(fd - gp[j]) <= 1e-5 * max(abs(gp[j]), 1e-3 * chi2 * h)
    hit = np.flatnonzero(np.bincount(pix.ravel(), minlength=obs.npix) > 10)
    for p in hit[:: max(1, hit.size // 6)][:6]:
        for k in range(3):
            hm = 1e-3
            mp = m.copy(); mp[p, k] += hm
            mm = m.copy(); mm[p, k] -= hm
            fd = (_chi2(orc, obs, delta, mp, d, nz) - _chi2(orc, obs, delta, mm, d, nz)) / (2 * hm)
            # chi^2 is quadratic in m: central differences are exact up to rounding
            assert abs(fd - gm[p, k]) <= 1e-6 * abs(gm[p, k]) + 1e-9 * chi2 / hm
