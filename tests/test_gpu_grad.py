"""chi^2 and its hand-written gradients (map and per-detector angle offsets) vs the oracle,
finite differences, and the torch.autograd.Function wrapper."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c5(orc):
    """Reduced config 5: nside 64, 8 detectors x 16384 samples, offsets ~ N(0, 1 deg)."""
    nd, ns = 8, 16384
    o = synth.Observation(64, synth.satellite_scan(ns, t0=200.0), synth.hex_focal_plane(nd))
    g = synth.rng(5, 3)
    dtrue = np.radians(g.normal(0, 1.0, nd))
    sky = synth.gaussian_sky(o.nside, g)
    taps = np.tile(synth.inverse_noise_taps(), (nd, 1))
    pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det, dtrue)
    d = orc.P(pix, c, s, sky) + synth.one_over_f_noise(nd, ns, g)
    return o, sky, taps, dtrue, d


def _oracle(orc, o, taps, delta, m, d):
    pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det, delta)
    return orc.chi2_grad(o.npix, pix, c, s, orc.Noise(taps=taps), m, d)


@pytest.mark.parametrize("precision,tol", [("f64", 1e-10), ("f32x2", 1e-10), ("f32", 1e-4)])
def test_chi2_grad_matches_oracle(fx, dev, orc, c5, precision, tol):
    o, sky, taps, dtrue, d = c5
    delta = dtrue / 2
    m = sky * 1.01
    chi2, gm, gp = _oracle(orc, o, taps, delta, m, d)
    o.psi_offset = delta
    P = fx.Pointing.from_observations([o], mode="cache_f64", device=dev)
    N = fx.Noise.banded(P, taps)
    dd = torch.as_tensor(d.ravel(), device=dev)
    if precision == "f32":
        dd = dd.float()
    c2, gmap, gpsi = fx.chi2_grad(P, N, dd, torch.as_tensor(m, device=dev), precision)
    assert abs(c2.item() - chi2) <= tol * chi2
    assert np.linalg.norm(gmap.cpu().numpy() - gm) <= tol * np.linalg.norm(gm) * 10
    assert np.max(np.abs(gpsi.cpu().numpy() - gp)) <= tol * np.max(np.abs(gp)) * 10
    o.psi_offset = None


def test_autograd_function_and_finite_differences(fx, dev, orc, c5):
    o, sky, taps, dtrue, d = c5
    P = fx.Pointing.from_observations([o], mode="on_the_fly", device=dev)
    N = fx.Noise.banded(P, taps)
    dd = torch.as_tensor(d.ravel(), device=dev)
    m = torch.as_tensor(sky * 1.01, device=dev).requires_grad_(True)
    delta = torch.as_tensor(dtrue / 2, device=dev).requires_grad_(True)
    val = fx.chi2(m, delta, P, N, dd)
    gm, gd = torch.autograd.grad(val, (m, delta))
    chi2, rgm, rgp = _oracle(orc, o, taps, dtrue / 2, sky * 1.01, d)
    assert abs(val.item() - chi2) <= 1e-10 * chi2
    np.testing.assert_allclose(gd.cpu().numpy(), rgp, rtol=1e-8, atol=1e-10 * np.abs(rgp).max())
    # central differences in delta on the GPU chi^2 (h = 1e-6 rad, FP64)
    h = 1e-6
    for j in range(0, 8, 3):
        e = torch.zeros(8, dtype=torch.float64, device=dev)
        e[j] = h
        with torch.no_grad():
            fp = fx.chi2(m, delta + e, P, N, dd).item()
            fm = fx.chi2(m, delta - e, P, N, dd).item()
        fd = (fp - fm) / (2 * h)
        assert abs(fd - gd[j].item()) <= 1e-5 * max(abs(gd[j].item()), 1e-3 * chi2 * h)


@pytest.mark.parametrize("mode", ["on_the_fly", "cache_mixed"])
@pytest.mark.parametrize("noise", ["banded", "white"])
def test_chi2_grad_double_fp32_and_fp32_across_modes(fx, dev, orc, c5, mode, noise):
    """The double-FP32 χ² and gradients (FP64-accurate weights: on the fly or the mixed cache)
    match the oracle to FP64-like accuracy, and the FP32 ones to FP32 accuracy, for a band and for
    white noise."""
    o, sky, taps, dtrue, d = c5
    delta = dtrue / 2
    m = sky * 1.01
    sigma2 = np.linspace(0.5, 1.5, o.ndet)
    on = orc.Noise(taps=taps) if noise == "banded" else orc.Noise(sigma2=sigma2)
    pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det, delta)
    chi2, gm, gp = orc.chi2_grad(o.npix, pix, c, s, on, m, d)
    o.psi_offset = delta
    P = fx.Pointing.from_observations([o], mode=mode, device=dev)
    N = fx.Noise.banded(P, taps) if noise == "banded" else fx.Noise.white(P, sigma2)
    dd = torch.as_tensor(d.ravel(), device=dev)
    for precision, tol, data in (("f32x2", 1e-10, dd), ("f32", 1e-4, dd.float())):
        c2, gmap, gpsi = fx.chi2_grad(P, N, data, torch.as_tensor(m, device=dev), precision)
        assert abs(c2.item() - chi2) <= tol * chi2, precision
        assert np.linalg.norm(gmap.cpu().numpy() - gm) <= tol * np.linalg.norm(gm) * 10, precision
        assert np.max(np.abs(gpsi.cpu().numpy() - gp)) <= tol * np.max(np.abs(gp)) * 10, precision
    o.psi_offset = None
