"""Pins for the oracle's geometry: quaternions, azimuth, HEALPix RING lookup, weights.

Each check compares the oracle with something other than itself: scipy rotations,
numpy's arctan2, the closed-form HEALPix ring layout (Gorski et al. 2005), an
independent pixel lookup through the HEALPix projection plane (Calabretta &
Roukema 2007), equal-area counting, and geometric identities of the polarisation
angle.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import synth


def _xyzw(q):
    return np.asarray(q)[:, [1, 2, 3, 0]]


def _random_unit_quats(n, seed):
    g = np.random.default_rng(seed)
    q = g.normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


# ---------------------------------------------------------------- quaternions
def test_quat_mul_matches_scipy_composition(orc):
    a = _random_unit_quats(2000, 1)
    b = _random_unit_quats(2000, 2)
    q = orc.quat_mul(a, b)
    ref = (Rotation.from_quat(_xyzw(a)) * Rotation.from_quat(_xyzw(b))).as_quat()
    ref = ref[:, [3, 0, 1, 2]]
    sign = np.sign(np.sum(ref * q, axis=1))[:, None]
    assert np.max(np.abs(q - sign * ref)) < 1e-15


def test_axes_match_scipy_rotation_columns(orc):
    q = _random_unit_quats(2000, 3)
    d, o = orc.quat_axes(q)
    r = Rotation.from_quat(_xyzw(q))
    assert np.max(np.abs(d - r.apply([0.0, 0.0, 1.0]))) < 2e-15
    assert np.max(np.abs(o - r.apply([1.0, 0.0, 0.0]))) < 2e-15


def test_axes_orthonormal_and_identity(orc):
    q = _random_unit_quats(5000, 4)
    d, o = orc.quat_axes(q)
    assert np.max(np.abs(np.linalg.norm(d, axis=1) - 1)) < 4e-16 * 4
    assert np.max(np.abs(np.linalg.norm(o, axis=1) - 1)) < 4e-16 * 4
    assert np.max(np.abs(np.sum(d * o, axis=1))) < 4e-16 * 4
    d, o = orc.quat_axes(np.array([[1.0, 0, 0, 0]]))
    assert np.array_equal(d[0], [0, 0, 1]) and np.array_equal(o[0], [1, 0, 0])


def test_composition_order_is_boresight_then_detector(orc):
    """q = q_bore (x) q_det applies the detector offset in the boresight frame."""
    qb = synth.satellite_scan(64)
    qd = synth.hex_focal_plane(7)[3:4]
    d, _ = orc.quat_axes(orc.quat_mul(qb, np.repeat(qd, 64, axis=0)))
    ref = (Rotation.from_quat(_xyzw(qb)) * Rotation.from_quat(_xyzw(qd))).apply([0, 0, 1.0])
    assert np.max(np.abs(d - ref)) < 2e-15


# ---------------------------------------------------------------- azimuth
def test_phi_close_to_libm_atan2(orc):
    g = np.random.default_rng(5)
    x = g.normal(size=200000) * 10.0 ** g.uniform(-8, 3, 200000)
    y = g.normal(size=200000) * 10.0 ** g.uniform(-8, 3, 200000)
    ph = orc.phi(x, y)
    ref = np.mod(np.arctan2(y, x), 2 * np.pi)
    ref = np.where(ref >= 2 * np.pi, 0.0, ref)
    ulp = np.spacing(np.maximum(np.abs(ref), 1e-300))
    err = np.abs(ph - ref)
    # compare modulo 2 pi (a value just below 2 pi and 0 are the same direction)
    err = np.minimum(err, np.abs(err - 2 * np.pi))
    assert np.all(err <= 4 * ulp + 1e-300)
    assert np.all((ph >= 0) & (ph < 2 * np.pi))


def test_phi_special_angles(orc):
    pi = math.pi
    vals = orc.phi([1.0, 0.0, -1.0, 0.0, 1.0, -2.0, 0.0, 3.0], [0.0, 1.0, 0.0, -1.0, 1.0, 2.0, 0.0, -3.0])
    assert vals[0] == 0.0
    assert vals[1] == pi / 2
    assert vals[2] == pi
    assert vals[3] == 2 * pi - pi / 2
    assert vals[4] == pi / 4
    assert vals[5] == pi - pi / 4
    assert vals[6] == 0.0
    assert vals[7] == 2 * pi - pi / 4


# ---------------------------------------------------------------- HEALPix RING
NSIDES = [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024]


@pytest.mark.parametrize("nside", NSIDES)
def test_poles_closed_form(orc, nside):
    npix = 12 * nside * nside
    assert orc.ang2pix(nside, [1.0], [0.0])[0] == 0
    assert orc.ang2pix(nside, [-1.0], [0.0])[0] == npix - 4
    assert orc.vec2pix(nside, [[0.0, 0.0, 1.0]])[0] == 0
    assert orc.vec2pix(nside, [[0.0, 0.0, -1.0]])[0] == npix - 4


def test_base_pixel_centres_nside1(orc):
    """Nside 1: three rings of four base pixels at z = 2/3, 0, -2/3."""
    z, ph = orc.pix2ang(1, np.arange(12))
    np.testing.assert_allclose(z, np.repeat([2 / 3, 0.0, -2 / 3], 4), atol=1e-15)
    np.testing.assert_allclose(ph, np.array([1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7]) * np.pi / 4, atol=1e-15)


@pytest.mark.parametrize("nside", NSIDES)
def test_round_trip_every_pixel(orc, nside):
    p = np.arange(12 * nside * nside, dtype=np.int64)
    z, ph = orc.pix2ang(nside, p)
    assert np.array_equal(orc.ang2pix(nside, z, ph), p)
    if nside <= 256:
        st = np.sqrt((1 - z) * (1 + z))
        v = np.stack([st * np.cos(ph), st * np.sin(ph), z], axis=1)
        assert np.array_equal(orc.vec2pix(nside, v), p)


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16, 64])
def test_ring_structure(orc, nside):
    """Ring i holds 4 min(i, N, 4N-i) pixels at z_i (caps 1 - i^2/3N^2, belt 4/3 - 2i/3N), evenly in phi."""
    n = nside
    z, ph = orc.pix2ang(n, np.arange(12 * n * n))
    start = 0
    for i in range(1, 4 * n):
        cnt = 4 * min(i, n, 4 * n - i)
        if i < n:
            zi = 1 - i * i / (3 * n * n)
        elif i <= 3 * n:
            zi = 4 / 3 - 2 * i / (3 * n)
        else:
            j = 4 * n - i
            zi = -(1 - j * j / (3 * n * n))
        zz = z[start:start + cnt]
        pp = ph[start:start + cnt]
        np.testing.assert_allclose(zz, zi, atol=2e-15)
        np.testing.assert_allclose(np.diff(pp), 2 * np.pi / cnt, rtol=1e-12)
        assert pp[0] < 2 * np.pi / cnt + 1e-12
        start += cnt
    assert start == 12 * n * n


def _projection_plane_lookup(nside, z, phi):
    """Independent RING lookup through the HEALPix projection (H=4, K=3; Calabretta & Roukema 2007).

    In the projection plane every pixel is a square of the lattice U = X - Y, V = X + Y
    (spacing 1/N); its centre gives ring 2N(1 - Yc) and the azimuth of the centre
    gives the position in the ring.
    """
    n = nside
    X = 2 * phi / np.pi
    za = np.abs(z)
    polar = za > 2 / 3
    sig = np.sqrt(3 * (1 - za))
    f = np.minimum(np.floor(X), 3)
    Xp = np.where(polar, f + 0.5 + (X - f - 0.5) * sig, X)
    Y = np.where(polar, np.sign(z) * (1 - sig / 2), 0.75 * z)
    iu = np.floor(n * (Xp - Y + 0.5))
    iv = np.floor(n * (Xp + Y + 0.5))
    Uc = (iu + 0.5) / n - 0.5
    Vc = (iv + 0.5) / n - 0.5
    Xc = (Uc + Vc) / 2
    Yc = (Vc - Uc) / 2
    ring = np.rint(2 * n * (1 - Yc)).astype(np.int64)
    out = np.empty(z.shape, np.int64)
    belt = (ring >= n) & (ring <= 3 * n)
    # belt: 4N pixels, centres at X = (k + shift)/N, shift 1/2 when ring - N is even
    shift = np.where((ring - n) % 2 == 0, 0.5, 0.0)
    k = np.mod(np.rint(Xc * n - shift).astype(np.int64), 4 * n)
    ncap = 2 * n * (n - 1)
    out[belt] = (ncap + (ring - n) * 4 * n + k)[belt]
    # caps: ring i' from its pole has 4 i' pixels at X = (k + 1/2)/i'; undo the facet compression
    ip = np.where(ring < n, ring, 4 * n - ring)
    sc = np.maximum(ip, 1) / n
    fc = np.floor(Xc)
    Xu = fc + 0.5 + (Xc - fc - 0.5) / sc
    kc = np.mod(np.rint(Xu * ip - 0.5).astype(np.int64), 4 * np.maximum(ip, 1))
    north = ring < n
    south = ring > 3 * n
    out[north] = (2 * ip * (ip - 1) + kc)[north]
    out[south] = (12 * n * n - 2 * ip * (ip + 1) + kc)[south]
    return out


@pytest.mark.parametrize("nside", [1, 2, 3, 4, 5, 8])
def test_projection_plane_lookup_agrees(orc, nside):
    g = np.random.default_rng(100 + nside)
    n = 1_000_000
    z = g.uniform(-1, 1, n)
    phi = g.uniform(0, 2 * np.pi, n)
    ref = _projection_plane_lookup(nside, z, phi)
    got = orc.ang2pix(nside, z, phi)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("nside", [4, 32])
def test_equal_area(orc, nside):
    """Uniform directions fall evenly into the 12 N^2 equal-area pixels (chi^2 test)."""
    g = np.random.default_rng(7 + nside)
    n = 10_000_000
    v = g.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    pix = orc.vec2pix(nside, v)
    npix = 12 * nside * nside
    counts = np.bincount(pix, minlength=npix)
    assert counts.size == npix
    e = n / npix
    chi2 = np.sum((counts - e) ** 2 / e)
    dof = npix - 1
    assert abs(chi2 - dof) < 6 * math.sqrt(2 * dof)


def test_vec2pix_matches_angle_form_off_edges(orc):
    """The cancellation-free cap formula picks the same pixel as the (z, phi) form."""
    g = np.random.default_rng(11)
    v = g.normal(size=(500000, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    for nside in (16, 512):
        a = orc.vec2pix(nside, v)
        b = orc.ang2pix(nside, v[:, 2], orc.phi(v[:, 0], v[:, 1]))
        # the two forms of 1-|z| differ by rounding only; disagreements need a point within
        # ~1e-15 of an edge, which uniform draws of this size do not produce
        assert np.array_equal(a, b)


# ---------------------------------------------------------------- polarisation weights
def _rz(alpha):
    return synth.copointed_detectors(np.degrees(np.atleast_1d(alpha)))


def _off_pole(orc, qb, qd, eps=1e-8):
    """[ndet][nsamp] mask of samples whose line of sight is not within eps of a pole."""
    ns, nd = qb.shape[0], qd.shape[0]
    q = orc.quat_mul(np.tile(qb, (nd, 1)), np.repeat(qd, ns, axis=0))
    d, _ = orc.quat_axes(q)
    return (d[:, 0] ** 2 + d[:, 1] ** 2 > eps).reshape(nd, ns)


def test_weights_unit_norm(orc):
    qb = synth.satellite_scan(4096)
    qd = synth.hex_focal_plane(19)
    pix, c, s, bad = orc.pointing(64, qb, qd)
    assert bad == 0
    assert np.max(np.abs(c * c + s * s - 1)) < 4e-16 * 4


def test_rotation_about_line_of_sight_shifts_psi(orc):
    """Turning the detector by +alpha about its line of sight (x towards y of the
    detector frame) turns its orientation from north towards west, so psi -> psi - alpha;
    the pixel is unchanged."""
    qb = synth.satellite_scan(2048)
    qd = synth.hex_focal_plane(7)
    alpha = 0.3141
    qd2 = orc.quat_mul(qd, np.repeat(_rz(alpha), qd.shape[0], axis=0))
    p1, c1, s1, _ = orc.pointing(256, qb, qd)
    p2, c2, s2, _ = orc.pointing(256, qb, qd2)
    assert np.array_equal(p1, p2)
    # psi is undefined exactly at a pole (the scan's first sample puts one detector there)
    ok = _off_pole(orc, qb, qd)
    assert ok.mean() > 0.999
    ca, sa = math.cos(-2 * alpha), math.sin(-2 * alpha)
    np.testing.assert_allclose(c2[ok], (c1 * ca - s1 * sa)[ok], atol=2e-14)
    np.testing.assert_allclose(s2[ok], (s1 * ca + c1 * sa)[ok], atol=2e-14)


def test_psi_offset_equals_detector_rotation(orc):
    qb = synth.satellite_scan(2048)
    qd = synth.hex_focal_plane(5)
    delta = np.array([0.01, -0.02, 0.3, 0.0, -1.1])
    p1, c1, s1, _ = orc.pointing(128, qb, qd, psi_offset=delta)
    qd2 = orc.quat_mul(qd, _rz(-delta))
    p2, c2, s2, _ = orc.pointing(128, qb, qd2)
    ok = _off_pole(orc, qb, qd)
    assert np.array_equal(p1[ok], p2[ok])
    np.testing.assert_allclose(c1[ok], c2[ok], atol=2e-14)
    np.testing.assert_allclose(s1[ok], s2[ok], atol=2e-14)


def test_psi_on_equator_closed_form(orc):
    """Line of sight x^ (theta = 90 deg, phi = 0): north is +z, east is +y. A detector whose
    x axis points to +z has psi = 0; one whose x axis points to +y (east) has psi = 90 deg."""
    # rotation taking z^ -> x^ and x^ -> z^ : quaternion of a rotation by pi about (x+z)/sqrt 2
    q_north = np.array([[0.0, 1 / math.sqrt(2), 0.0, 1 / math.sqrt(2)]])
    # z^ -> x^, x^ -> y^ : cyclic permutation (rotation by 120 deg about (1,1,1))
    q_east = np.array([[0.5, 0.5, 0.5, 0.5]])
    one = np.array([[1.0, 0, 0, 0]])
    for q, (ce, se) in ((q_north, (1.0, 0.0)), (q_east, (-1.0, 0.0))):
        d, o = orc.quat_axes(q)
        np.testing.assert_allclose(d[0], [1, 0, 0], atol=1e-15)
        _, c, s, _ = orc.pointing(8, q, one)
        np.testing.assert_allclose([c[0, 0], s[0, 0]], [ce, se], atol=1e-15)
    # 45 deg between north and east: sin 2 psi = 1
    q45 = orc.quat_mul(q_north, _rz(-math.pi / 4))
    _, c, s, _ = orc.pointing(8, q45, one)
    np.testing.assert_allclose([c[0, 0], s[0, 0]], [0.0, 1.0], atol=1e-15)


def test_nonfinite_quaternion_gives_invalid_pixel(orc):
    qb = synth.satellite_scan(16)
    qb[5, 2] = np.nan
    qb[9, 0] = np.inf
    pix, c, s, bad = orc.pointing(16, qb, synth.copointed_detectors([0.0, 45.0]))
    assert bad == 4
    assert np.all(pix[:, [5, 9]] == -1)
    assert np.all(c[:, [5, 9]] == 0) and np.all(s[:, [5, 9]] == 0)


def test_far_from_unit_quaternion_never_leaves_the_map(orc):
    """Quaternions of norm up to 3 can push the cap formula past the last ring; such samples
    get pixel -1, every other pixel stays inside the map."""
    qb = synth.satellite_scan(20000) * np.linspace(0.3, 3.0, 20000)[:, None]
    pix, c, s, bad = orc.pointing(64, qb, synth.copointed_detectors([0.0, 45.0]))
    assert np.all((pix == -1) | ((pix >= 0) & (pix < 12 * 64 * 64)))
    assert bad == (pix == -1).sum() and bad > 0
    assert np.all(c[pix == -1] == 0)
