"""Pins for the template-deprojection oracle (F_T = W - W T (T^T W T)^-1 T^T W, Statement of
Need; TemplateOperator, Table 3): textbook and library routines, identities of the operator,
and dense brute force on tiny problems. Nothing here calls the oracle's own formula twice."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly
from scipy.linalg import toeplitz

import oracle
import synth
from oracle import templates as ot


def band_matrix(taps, ns):
    """Dense symmetric Toeplitz W with W[t, s] = c_|t-s| for |t-s| < K, truncated to the stream."""
    col = np.zeros(ns)
    k = min(len(taps), ns)
    col[:k] = taps[:k]
    return toeplitz(col)


@pytest.fixture(scope="module")
def lib():
    oracle.build()
    return oracle


@pytest.mark.parametrize("ns", [1, 2, 5, 64, 1001])
@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_legendre_columns_match_numpy(ns, order):
    if ns < order + 1 and ns > 1:
        pytest.skip("fewer samples than templates")
    T = ot.legendre_templates(ns, order)
    tau = np.zeros(ns) if ns == 1 else np.linspace(-1.0, 1.0, ns)
    assert np.allclose(T, npleg.legvander(tau, order), rtol=0, atol=1e-14)
    closed = [np.ones(ns), tau, (3 * tau ** 2 - 1) / 2, (5 * tau ** 3 - 3 * tau) / 2]
    for l in range(order + 1):
        assert np.allclose(T[:, l], closed[l], rtol=0, atol=1e-14)


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_white_noise_deprojection_is_polyfit_residual(lib, order):
    """W = diag(1/sigma^2): F_T x = (x - least-squares polynomial of degree K) / sigma^2."""
    g = np.random.default_rng(3)
    nd, ns = 3, 257
    x = g.normal(size=(nd, ns)) + np.linspace(0, 5, ns) ** 2
    sigma2 = np.array([0.5, 2.0, 7.0])
    y = ot.deproject(oracle.Noise(sigma2=sigma2), order, x)
    t = np.arange(ns, dtype=np.float64)
    for i in range(nd):
        coef = nppoly.polyfit(t, x[i], order)
        ref = (x[i] - nppoly.polyval(t, coef)) / sigma2[i]
        assert np.allclose(y[i], ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    if order == 0:
        assert np.allclose(y, (x - x.mean(axis=1, keepdims=True)) / sigma2[:, None], atol=1e-12)


@pytest.mark.parametrize("ns", [40, 300])
@pytest.mark.parametrize("order", [0, 1, 3])
def test_templates_are_annihilated_and_operator_is_symmetric(lib, ns, order):
    """F_T T = 0 and <u, F_T v> = <F_T u, v> (banded W, streams shorter and longer than the band)."""
    taps = np.stack([synth.inverse_noise_taps(), 1.5 * synth.inverse_noise_taps()])
    noise = oracle.Noise(taps=taps)
    T = ot.legendre_templates(ns, order)
    for l in range(order + 1):
        y = ot.deproject(noise, order, np.tile(T[:, l], (2, 1)))
        scale = np.abs(noise.apply(np.tile(T[:, l], (2, 1)))).max()
        assert np.abs(y).max() < 1e-10 * scale
    g = np.random.default_rng(4)
    u, v = g.normal(size=(2, 2, ns))
    lhs = np.sum(u * ot.deproject(noise, order, v), axis=1)
    rhs = np.sum(ot.deproject(noise, order, u) * v, axis=1)
    assert np.allclose(lhs, rhs, rtol=1e-11, atol=0)


@pytest.mark.parametrize("ns,order", [(50, 2), (200, 3), (200, 0)])
def test_deprojection_matches_dense_matrices(lib, ns, order):
    """Dense W (Toeplitz band), T (numpy Legendre basis): F_T = W - W T (T^T W T)^-1 T^T W, and
    F_T W^-1 F_T = F_T."""
    taps = synth.inverse_noise_taps()
    noise = oracle.Noise(taps=taps[None, :])
    W = band_matrix(taps, ns)
    T = npleg.legvander(np.linspace(-1, 1, ns), order)
    G = T.T @ W @ T
    F = W - W @ T @ np.linalg.solve(G, T.T @ W)
    assert np.allclose(ot.gram(noise, 1, ns, order)[0], G, rtol=1e-11, atol=1e-11 * np.abs(G).max())
    x = np.random.default_rng(5).normal(size=(1, ns))
    y = ot.deproject(noise, order, x)[0]
    assert np.allclose(y, F @ x[0], rtol=0, atol=1e-10 * np.abs(F @ x[0]).max())
    FWF = F @ np.linalg.solve(W, F)
    assert np.allclose(FWF, F, rtol=0, atol=1e-8 * np.abs(F).max())


def dense_pointing(npix, pix, c, s):
    """Dense P [ndet*ns][3*npix] (invalid samples: zero rows)."""
    nd, ns = pix.shape
    Pm = np.zeros((nd * ns, 3 * npix))
    for i in range(nd):
        for t in range(ns):
            p = pix[i, t]
            if p >= 0:
                Pm[i * ns + t, 3 * p:3 * p + 3] = (1.0, c[i, t], s[i, t])
    return Pm


@pytest.fixture(scope="module")
def tiny(lib):
    o = synth.Observation(2, synth.satellite_scan(180, t0=20.0), synth.hex_focal_plane(4))
    pix, c, s, _ = oracle.pointing(o.nside, o.q_bore, o.q_det)
    taps = np.tile(synth.inverse_noise_taps(), (4, 1)) * np.array([1.0, 1.3, 0.8, 1.1])[:, None]
    return o, pix, c, s, oracle.Noise(taps=taps), taps


@pytest.mark.parametrize("order", [0, 2])
def test_normal_operator_matches_dense(tiny, order):
    o, pix, c, s, noise, taps = tiny
    nd, ns = pix.shape
    Pm = dense_pointing(o.npix, pix, c, s)
    Fb = np.zeros((nd * ns, nd * ns))
    T = npleg.legvander(np.linspace(-1, 1, ns), order)
    for i in range(nd):
        W = band_matrix(taps[i], ns)
        Fb[i * ns:(i + 1) * ns, i * ns:(i + 1) * ns] = W - W @ T @ np.linalg.solve(T.T @ W @ T, T.T @ W)
    A = Pm.T @ Fb @ Pm
    g = np.random.default_rng(6)
    x = g.normal(size=(o.npix, 3))
    valid = g.random(o.npix) > 0.2
    xm = np.where(valid[:, None], x, 0.0)
    ref = np.where(valid[:, None], (A @ xm.ravel()).reshape(-1, 3), 0.0)
    got = ot.ptfp_apply(o.npix, pix, c, s, noise, order, valid, x)
    assert np.allclose(got, ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    d = g.normal(size=(nd, ns))
    rref = np.where(valid[:, None], (Pm.T @ Fb @ d.ravel()).reshape(-1, 3), 0.0)
    assert np.allclose(ot.rhs(o.npix, pix, c, s, noise, order, valid, d), rref, rtol=0,
                       atol=1e-10 * np.abs(rref).max())


def test_estimator_is_invariant_under_template_contamination(tiny):
    """d -> d + T alpha leaves the right-hand side and the solved map unchanged."""
    o, pix, c, s, noise, _ = tiny
    nd, ns = pix.shape
    order = 2
    g = np.random.default_rng(7)
    sky = synth.gaussian_sky(o.nside, g)
    d = oracle.P(pix, c, s, sky) + g.normal(size=(nd, ns)) * 0.1
    alpha = g.normal(size=(nd, order + 1)) * 50.0
    d2 = d + alpha @ ot.legendre_templates(ns, order).T
    bjd = oracle.bj(o.npix, pix, c, s, noise, rcond_min=1e-6)
    b1 = ot.rhs(o.npix, pix, c, s, noise, order, bjd["valid"], d)
    b2 = ot.rhs(o.npix, pix, c, s, noise, order, bjd["valid"], d2)
    assert np.allclose(b1, b2, rtol=0, atol=1e-9 * np.abs(b1).max())
    x1, _, _ = ot.pcg(o.npix, pix, c, s, noise, order, bjd["valid"], bjd["inv"], b1, 200, 1e-12)
    x2, _, _ = ot.pcg(o.npix, pix, c, s, noise, order, bjd["valid"], bjd["inv"], b2, 200, 1e-12)
    assert np.allclose(x1, x2, rtol=0, atol=1e-7 * np.abs(x1).max())


def test_pcg_solves_the_dense_normal_equations(tiny):
    """The PCG limit solves the dense system; with offset templates the I monopole of the
    observed pixels is the (near-)null direction, so maps are compared with it removed."""
    o, pix, c, s, noise, taps = tiny
    nd, ns = pix.shape
    order = 1
    bjd = oracle.bj(o.npix, pix, c, s, noise, rcond_min=1e-6)
    v = bjd["valid"]
    g = np.random.default_rng(8)
    d = oracle.P(pix, c, s, synth.gaussian_sky(o.nside, g)) + g.normal(size=(nd, ns))
    b = ot.rhs(o.npix, pix, c, s, noise, order, v, d)
    x, it, hist = ot.pcg(o.npix, pix, c, s, noise, order, v, bjd["inv"], b, 400, 1e-11)
    assert hist[-1] <= 1e-11
    Pm = dense_pointing(o.npix, pix, c, s)
    Fb = np.zeros((nd * ns, nd * ns))
    T = npleg.legvander(np.linspace(-1, 1, ns), order)
    for i in range(nd):
        W = band_matrix(taps[i], ns)
        Fb[i * ns:(i + 1) * ns, i * ns:(i + 1) * ns] = W - W @ T @ np.linalg.solve(T.T @ W @ T, T.T @ W)
    cols = np.repeat(v, 3)
    A = (Pm.T @ Fb @ Pm)[np.ix_(cols, cols)]
    bd = (Pm.T @ Fb @ d.ravel())[cols]
    xd = np.linalg.lstsq(A, bd, rcond=1e-12)[0].reshape(-1, 3)
    xs = x[v]
    for m in (xs, xd):
        m[:, 0] -= m[:, 0].mean()
    assert np.allclose(xs, xd, rtol=0, atol=1e-6 * np.abs(xd).max())
