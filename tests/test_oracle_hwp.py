"""Oracle pins for HWP-modulated pointing (ideal half-wave plate, HWPOperator in Table 3 of the
Furax paper; commutation rule R(theta) o HWP = HWP o R(-theta) in "Algebraic reductions").

With a plate at angle w in front of a detector whose polarisation angle is psi (offset delta
included) the weights are (1, cos(4w - 2psi), sin(4w - 2psi)); the pixel does not change."""
import math

import numpy as np

import synth


def _psi(c, s):
    return 0.5 * np.arctan2(s, c)


def test_zero_angle_flips_u(orc):
    o = synth.Observation(16, synth.satellite_scan(3000), synth.hex_focal_plane(5))
    pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det)
    pix2, c2, s2, _ = orc.pointing(o.nside, o.q_bore, o.q_det, hwp=np.zeros(3000))
    assert np.array_equal(pix, pix2)
    assert np.array_equal(c2, c) and np.array_equal(s2, -s)      # 1 c + 0 s, 0 c - 1 s: exact


def test_weights_match_angle_formula_with_offsets(orc):
    """Independent evaluation from angles: cos(4w - 2(psi + delta)), sin(...)."""
    o = synth.Observation(32, synth.satellite_scan(4000, t0=70.0), synth.hex_focal_plane(7))
    w = synth.hwp_angle(4000, omega0=0.3)
    delta = np.radians(np.linspace(-2.0, 3.0, 7))
    pix, c0, s0, _ = orc.pointing(o.nside, o.q_bore, o.q_det)
    pix2, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det, psi_offset=delta, hwp=w)
    assert np.array_equal(pix, pix2)
    ok = pix >= 0
    ang = 4 * w[None, :] - 2 * (_psi(c0, s0) + delta[:, None])
    np.testing.assert_allclose(c[ok], np.cos(ang)[ok], atol=2e-13)
    np.testing.assert_allclose(s[ok], np.sin(ang)[ok], atol=2e-13)
    np.testing.assert_allclose((c * c + s * s)[ok], 1.0, atol=4e-16 * 8)


def test_quarter_turn_periodicity(orc):
    """A plate turned by pi/2 gives the same weights (4w changes by 2 pi)."""
    o = synth.Observation(16, synth.satellite_scan(2000), synth.hex_focal_plane(3))
    w = synth.hwp_angle(2000)
    _, c1, s1, _ = orc.pointing(o.nside, o.q_bore, o.q_det, hwp=w)
    _, c2, s2, _ = orc.pointing(o.nside, o.q_bore, o.q_det, hwp=w + math.pi / 2)
    np.testing.assert_allclose(c2, c1, atol=1e-13)
    np.testing.assert_allclose(s2, s1, atol=1e-13)


def test_four_plate_angles_give_closed_form_block(orc):
    """One detector, a fixed line of sight and the plate at 0, pi/8, pi/4, 3pi/8: the weights'
    angles are spaced by pi/2, so the block is diag(4, 2, 2)/sigma^2 whatever psi is."""
    for psi_det in (0.0, 17.0, 61.0):
        q_bore = np.tile(np.array([[0.9, 0.1, -0.3, 0.2]]) / np.linalg.norm([0.9, 0.1, -0.3, 0.2]), (8, 1))
        w = np.array([0.0, math.pi / 8, math.pi / 4, 3 * math.pi / 8] * 2)
        pix, c, s, _ = orc.pointing(2, q_bore, synth.copointed_detectors([psi_det]), hwp=w)
        bj = orc.bj(48, pix, c, s, orc.Noise(sigma2=np.array([100.0])))
        p = pix[0, 0]
        assert np.all(pix == p) and bj["hits"][p] == 8 and bj["valid"][p]
        idx = np.array([[0, 1, 2], [1, 3, 4], [2, 4, 5]])
        np.testing.assert_allclose(bj["blocks"][p][idx], np.diag([8.0, 4.0, 4.0]) / 100.0, atol=1e-15)
        np.testing.assert_allclose(bj["rcond"][p], 0.5, rtol=1e-12)


def test_single_detector_recovers_iqu(orc):
    """A rotating plate lets one detector measure Q and U: from noiseless data the binned map
    equals the input sky on every valid pixel."""
    o = synth.Observation(8, synth.satellite_scan(20000), synth.copointed_detectors([0.0]))
    w = synth.hwp_angle(20000)
    pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det, hwp=w)
    sky = synth.gaussian_sky(o.nside, synth.rng(9, 0))
    nz = orc.Noise(sigma2=np.array([100.0]))
    bj = orc.bj(o.npix, pix, c, s, nz)
    v = bj["valid"]
    assert v.sum() > 0.5 * (bj["hits"] > 0).sum()
    b = orc.rhs(o.npix, pix, c, s, nz, v, orc.P(pix, c, s, sky))
    m = orc.binned_map(bj, b)
    np.testing.assert_allclose(m[v], sky[v], rtol=0, atol=1e-9 * np.abs(sky).max())
    # without the plate the same single detector cannot separate Q from U: no pixel is valid
    pix0, c0, s0, _ = orc.pointing(o.nside, o.q_bore, o.q_det)
    assert orc.bj(o.npix, pix0, c0, s0, nz)["valid"].sum() < v.sum()


def test_offset_gradient_sign_finite_differences(orc):
    """d chi^2 / d delta with the plate: central finite differences of the oracle's chi^2."""
    nd, ns = 3, 3000
    o = synth.Observation(8, synth.satellite_scan(ns), synth.hex_focal_plane(nd))
    w = synth.hwp_angle(ns, omega0=0.1)
    delta = np.radians([0.4, -0.7, 1.1])
    sky = synth.gaussian_sky(o.nside, synth.rng(9, 1))
    pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det, psi_offset=np.radians([1.0, 0.5, -0.3]), hwp=w)
    d = orc.P(pix, c, s, sky) + synth.white_noise(nd, ns, synth.rng(9, 2))
    nz = orc.Noise(taps=np.tile(synth.inverse_noise_taps(), (nd, 1)))
    pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det, psi_offset=delta, hwp=w)
    _, _, gp = orc.chi2_grad(o.npix, pix, c, s, nz, sky, d, hwp=True)
    h = 1e-6
    for j in range(nd):
        dp = delta.copy(); dp[j] += h
        dm = delta.copy(); dm[j] -= h
        _, cp, sp, _ = orc.pointing(o.nside, o.q_bore, o.q_det, psi_offset=dp, hwp=w)
        _, cm, sm, _ = orc.pointing(o.nside, o.q_bore, o.q_det, psi_offset=dm, hwp=w)
        fp, _, _ = orc.chi2_grad(o.npix, pix, cp, sp, nz, sky, d, want_grad=False)
        fm, _, _ = orc.chi2_grad(o.npix, pix, cm, sm, nz, sky, d, want_grad=False)
        fd = (fp - fm) / (2 * h)
        assert abs(fd - gp[j]) <= 1e-5 * max(abs(gp[j]), 1.0), (j, fd, gp[j])
