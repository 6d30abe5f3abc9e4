"""Pins for the oracle's operators: P, P^T, hits, N^-1 (white, banded), block-Jacobi."""
import math

import numpy as np
import pytest
import scipy.linalg

import synth


@pytest.fixture(scope="module")
def c1_small(orc):
    obs, sky, noise, sigma2 = synth.config1(nsamp=16384, nside=16)
    pix, c, s, bad = orc.pointing(obs.nside, obs.q_bore, obs.q_det)
    assert bad == 0
    return obs, sky, noise, sigma2, pix, c, s


@pytest.fixture(scope="module")
def hex_small(orc):
    obs = synth.Observation(8, synth.satellite_scan(8192), synth.hex_focal_plane(16))
    pix, c, s, bad = orc.pointing(obs.nside, obs.q_bore, obs.q_det)
    assert bad == 0
    return obs, pix, c, s


# ---------------------------------------------------------------- P
def test_pair_differencing_identities(orc, c1_small):
    """Co-pointed detectors at 0/45/90/135 deg: d0 + d90 = 2I, d0 - d90 = 2Q', d45 - d135 = 2U'
    where (Q', U') is the sky (Q, U) rotated by -2 psi_boresight: I recovered exactly,
    and Q'^2 + U'^2 = Q^2 + U^2 (polarised intensity is frame independent)."""
    obs, sky, _, _, pix, c, s = c1_small
    tod = orc.P(pix, c, s, sky)
    p = pix[0]
    assert np.all(pix == p[None, :])
    np.testing.assert_allclose(0.5 * (tod[0] + tod[2]), sky[p, 0], rtol=0, atol=1e-12)
    np.testing.assert_allclose(0.5 * (tod[1] + tod[3]), sky[p, 0], rtol=0, atol=1e-12)
    qq = 0.5 * (tod[0] - tod[2])
    uu = 0.5 * (tod[1] - tod[3])
    np.testing.assert_allclose(qq ** 2 + uu ** 2, sky[p, 1] ** 2 + sky[p, 2] ** 2, rtol=1e-9, atol=1e-12)


def test_P_unpolarised_sky_is_gather(orc, hex_small):
    obs, pix, c, s = hex_small
    m = np.zeros((obs.npix, 3))
    m[:, 0] = np.arange(obs.npix) * 0.5
    tod = orc.P(pix, c, s, m)
    assert np.array_equal(tod, m[pix, 0])


def test_adjoint_identity(orc, hex_small):
    obs, pix, c, s = hex_small
    g = np.random.default_rng(1)
    m = g.normal(size=(obs.npix, 3))
    d = g.normal(size=pix.shape)
    lhs = np.dot(orc.P(pix, c, s, m).ravel(), d.ravel())
    mt, _ = orc.PT(obs.npix, pix, c, s, d)
    rhs = np.dot(m.ravel(), mt.ravel())
    assert abs(lhs - rhs) <= 1e-13 * (np.abs(orc.P(pix, c, s, m)).ravel() @ np.abs(d).ravel())


def test_hits_are_bincount(orc, hex_small):
    obs, pix, c, s = hex_small
    _, hits = orc.PT(obs.npix, pix, c, s, np.ones(pix.shape))
    assert np.array_equal(hits, np.bincount(pix.ravel(), minlength=obs.npix))


def test_PT_of_ones_counts_weights(orc, hex_small):
    """P^T 1 = (hits, sum c, sum s) per pixel; checked against bincount with weights."""
    obs, pix, c, s = hex_small
    m, hits = orc.PT(obs.npix, pix, c, s, np.ones(pix.shape))
    np.testing.assert_allclose(m[:, 0], hits, rtol=0, atol=0)
    np.testing.assert_allclose(m[:, 1], np.bincount(pix.ravel(), c.ravel(), obs.npix), atol=1e-11)
    np.testing.assert_allclose(m[:, 2], np.bincount(pix.ravel(), s.ravel(), obs.npix), atol=1e-11)


def test_PT_skips_invalid_samples(orc):
    pix = np.array([[0, -1, 2, -1]], np.int32)
    c = np.array([[1.0, 0.0, 0.5, 0.0]])
    s = np.array([[0.0, 0.0, 0.5, 0.0]])
    m, hits = orc.PT(3, pix, c, s, np.array([[1.0, 100.0, 2.0, 100.0]]))
    assert np.array_equal(hits, [1, 0, 1])
    np.testing.assert_array_equal(m, [[1, 1, 0], [0, 0, 0], [2, 1, 1]])
    tod = orc.P(pix, c, s, np.ones((3, 3)))
    np.testing.assert_array_equal(tod, [[2.0, 0.0, 2.0, 0.0]])


# ---------------------------------------------------------------- N^-1
def test_ninv_white(orc):
    g = np.random.default_rng(2)
    x = g.normal(size=(3, 100))
    s2 = np.array([4.0, 100.0, 0.25])
    np.testing.assert_allclose(orc.ninv_white(s2, x), x / s2[:, None], rtol=1e-16)


@pytest.mark.parametrize("ns", [1, 5, 63, 64, 65, 127, 300, 1000])
def test_band_matches_dense_toeplitz(orc, ns):
    taps = synth.inverse_noise_taps()
    g = np.random.default_rng(ns)
    x = g.normal(size=(2, ns))
    col = np.zeros(ns)
    k = min(ns, taps.size)
    col[:k] = taps[:k]
    T = scipy.linalg.toeplitz(col)
    y = orc.ninv_band(np.stack([taps, 2 * taps]), x)
    np.testing.assert_allclose(y[0], T @ x[0], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(y[1], 2 * (T @ x[1]), rtol=1e-12, atol=1e-15)


def test_band_matches_fft_circular_convolution_interior(orc):
    taps = synth.inverse_noise_taps()
    ns = 4096
    x = np.random.default_rng(3).normal(size=(1, ns))
    kern = np.zeros(ns)
    kern[:64] = taps
    kern[-63:] = taps[1:][::-1]
    ycirc = np.fft.irfft(np.fft.rfft(x[0]) * np.fft.rfft(kern), n=ns)
    y = orc.ninv_band(taps, x)[0]
    np.testing.assert_allclose(y[63:ns - 63], ycirc[63:ns - 63], rtol=1e-10, atol=1e-13)


def test_band_symmetric_and_positive_definite(orc):
    taps = synth.inverse_noise_taps()
    g = np.random.default_rng(4)
    x = g.normal(size=(1, 777)); y = g.normal(size=(1, 777))
    a = np.dot(x[0], orc.ninv_band(taps, y)[0])
    b = np.dot(orc.ninv_band(taps, x)[0], y[0])
    assert abs(a - b) < 1e-13 * max(abs(a), 1e-300) + 1e-16
    col = np.zeros(512); col[:64] = taps
    scipy.linalg.cholesky(scipy.linalg.toeplitz(col))  # raises if not SPD
    w = np.linspace(0, np.pi, 1 << 16)
    symbol = taps[0] + 2 * np.cos(np.outer(w, np.arange(1, 64))) @ taps[1:]
    assert symbol.min() > 0


def test_white_taps_reduce_to_homothety():
    """A flat PSD (no 1/f) makes the band a single tap 1/sigma^2 (N^-1 = sigma^-2 I), up to
    the removed zero-frequency bin, which shifts every lag by -1/(L sigma^2)."""
    L = 1 << 16
    taps = synth.inverse_noise_taps(fknee=0.0, nfft=L)
    np.testing.assert_allclose(taps[0], 1 / synth.SIGMA_UK ** 2, rtol=2.0 / L)
    assert np.max(np.abs(taps[1:])) <= 1.0001 / (L * synth.SIGMA_UK ** 2)


# ---------------------------------------------------------------- block-Jacobi
def test_bj_closed_form_copointed(orc, c1_small):
    """4 co-pointed detectors at 0/45/90/135 deg: sum w w^T = diag(4, 2, 2) per time sample,
    so M_p = (hits_p/4) diag(4, 2, 2)/sigma^2 and rcond = 1/2."""
    obs, _, _, sigma2, pix, c, s = c1_small
    bj = orc.bj(obs.npix, pix, c, s, orc.Noise(sigma2=sigma2))
    h = bj["hits"].astype(float)
    M = bj["blocks"]
    scale = h / 4 / synth.SIGMA_UK ** 2
    np.testing.assert_allclose(M[:, 0], 4 * scale, rtol=1e-13)
    np.testing.assert_allclose(M[:, 3], 2 * scale, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(M[:, 5], 2 * scale, rtol=1e-12, atol=1e-14)
    for k in (1, 2, 4):
        assert np.max(np.abs(M[:, k])) < 1e-12 * max(scale.max(), 1)
    hit = h >= 4
    np.testing.assert_allclose(bj["rcond"][hit], 0.5, rtol=1e-10)
    assert np.array_equal(bj["valid"], h >= 4)


def test_bj_inverse_spd_and_rcond(orc, hex_small):
    obs, pix, c, s = hex_small
    taps = np.tile(synth.inverse_noise_taps(), (pix.shape[0], 1))
    bj = orc.bj(obs.npix, pix, c, s, orc.Noise(taps=taps), rcond_min=1e-3)
    idx = np.array([[0, 1, 2], [1, 3, 4], [2, 4, 5]])
    M = bj["blocks"][:, idx]
    Minv = bj["inv"][:, idx]
    v = bj["valid"]
    assert v.sum() > 10
    np.testing.assert_allclose(np.einsum("pij,pjk->pik", M[v], Minv[v]), np.broadcast_to(np.eye(3), (v.sum(), 3, 3)), atol=1e-9)
    np.linalg.cholesky(M[v])
    rc = 1 / (np.linalg.norm(M[v], 1, axis=(1, 2)) * np.linalg.norm(np.linalg.inv(M[v]), 1, axis=(1, 2)))
    np.testing.assert_allclose(bj["rcond"][v], rc, rtol=1e-9)
    # the validity rule: at least 3 hits, positive definite, rcond >= threshold
    allrc = np.zeros(obs.npix)
    hitm = bj["hits"] >= 3
    ok = hitm & (np.linalg.eigvalsh(M)[:, 0] > 0)
    allrc[ok] = 1 / (np.linalg.norm(M[ok], 1, axis=(1, 2)) * np.linalg.norm(np.linalg.inv(M[ok]), 1, axis=(1, 2)))
    assert np.array_equal(v, ok & (allrc >= 1e-3))
    assert np.all(bj["inv"][~v] == 0)


def _blocks_from_samples(orc, angles_per_pixel, npix=12):
    """One detector whose samples visit pixel k at the polarisation angles angles_per_pixel[k]."""
    pix, c, s = [], [], []
    for k, angs in enumerate(angles_per_pixel):
        for a in angs:
            pix.append(k); c.append(math.cos(2 * a)); s.append(math.sin(2 * a))
    pix = np.array([pix], np.int32); c = np.array([c]); s = np.array([s])
    return orc.bj(npix, pix, c, s, orc.Noise(sigma2=np.array([100.0])), rcond_min=1e-3)


def test_bj_singular_blocks_are_invalid(orc):
    """A pixel crossed several times at one angle (or two) has a singular block: it must be
    excluded, never inverted. Well-spread angles give the textbook inverse."""
    bj = _blocks_from_samples(orc, [
        [0.3] * 4,                                   # rank 1
        [0.1, 0.1, 0.7, 0.7, 0.1],                  # rank 2
        [0.0, math.pi / 4, math.pi / 2, 3 * math.pi / 4],   # well conditioned: diag(4, 2, 2)/100
        [0.2, 1.1, 2.3],                             # three distinct angles: rank 3
        [0.5, 0.5000001, 0.4999999],                 # nearly one angle: rcond far below 1e-3
    ])
    assert list(bj["valid"][:5]) == [False, False, True, True, False]
    idx = np.array([[0, 1, 2], [1, 3, 4], [2, 4, 5]])
    for k in (2, 3):
        M = bj["blocks"][k][idx]
        np.testing.assert_allclose(bj["inv"][k][idx], np.linalg.inv(M), rtol=1e-12, atol=1e-14 * np.abs(np.linalg.inv(M)).max())
    np.testing.assert_allclose(bj["inv"][2][idx], np.diag([100 / 4, 100 / 2, 100 / 2]), rtol=1e-13, atol=1e-12)
    assert bj["rcond"][4] < 1e-3


def test_bj_precession_repeats(orc):
    """A scan longer than one precession period (72,000 samples at 20 Hz) crosses some pixels
    only at the same angle, one hour apart: their blocks are singular up to rounding. An inverse
    through the adjugate/determinant of such a block is noise and can pass an rcond test; the
    oracle's Cholesky inverse rejects them, and every accepted inverse is positive definite."""
    o = synth.Observation(256, synth.satellite_scan(160000), synth.hex_focal_plane(4))
    pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det)
    bj = orc.bj(o.npix, pix, c, s, orc.Noise(taps=np.tile(synth.inverse_noise_taps(), (4, 1))), rcond_min=1e-2)
    idx = np.array([[0, 1, 2], [1, 3, 4], [2, 4, 5]])
    M = bj["blocks"][:, idx]
    v = bj["valid"]
    assert np.all(np.linalg.eigvalsh(bj["inv"][v][:, idx])[:, 0] > 0)
    ev = np.linalg.eigvalsh(M)
    singular = (bj["hits"] >= 3) & (ev[:, 0] < 1e-12 * ev[:, 2])
    assert singular.sum() > 0                        # the case occurs in this scan
    assert not np.any(v & singular)
    # the adjugate/determinant rule would have accepted some of them with an indefinite inverse
    a, b_, c_, d, e, f = (bj["blocks"][:, k] for k in range(6))
    A_, B_, C_ = d * f - e * e, c_ * e - b_ * f, b_ * e - c_ * d
    det = a * A_ + b_ * B_ + c_ * C_
    adj = np.stack([A_, B_, C_, a * f - c_ * c_, b_ * c_ - a * e, a * d - b_ * b_], 1)
    sel = singular & (det > 0)
    if sel.any():
        inv_adj = adj[sel] / det[sel, None]
        rc = 1 / (np.linalg.norm(M[sel], 1, axis=(1, 2)) * np.linalg.norm(inv_adj[:, idx], 1, axis=(1, 2)))
        fooled = rc >= 1e-2
        assert fooled.any() and np.any(np.linalg.eigvalsh(inv_adj[fooled][:, idx])[:, 0] < 0)


def test_bj_blocks_equal_PT_diag_P(orc, hex_small):
    """M_p = P_p^T diag(N^-1) P_p: the block of the dense operator with the diagonal noise."""
    obs, pix, c, s = hex_small
    sig2 = np.linspace(50, 150, pix.shape[0])
    bj = orc.bj(obs.npix, pix, c, s, orc.Noise(sigma2=sig2))
    # dense P^T W P from unit maps, one column at a time, for a handful of pixels
    g = np.random.default_rng(9)
    for p in g.choice(np.flatnonzero(bj["hits"] > 0), 5, replace=False):
        cols = []
        for k in range(3):
            m = np.zeros((obs.npix, 3)); m[p, k] = 1.0
            t = orc.P(pix, c, s, m) / sig2[:, None]
            mt, _ = orc.PT(obs.npix, pix, c, s, t)
            cols.append(mt[p])
        dense = np.array(cols).T
        b = bj["blocks"][p]
        np.testing.assert_allclose(dense, [[b[0], b[1], b[2]], [b[1], b[3], b[4]], [b[2], b[4], b[5]]], rtol=1e-12, atol=1e-15)
