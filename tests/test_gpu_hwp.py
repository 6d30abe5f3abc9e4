"""HWP-modulated pointing on the GPU vs the oracle (ideal half-wave plate, HWPOperator in Table 3
of the Furax paper): pixels bit-exact, weights (1, cos(4w - 2psi), sin(4w - 2psi)) with and without
per-detector offsets (the GPU passes the offsets through the plate with the paper's commutation
rule, the oracle applies the definition), the normal operator, a single-detector solve that needs
the plate, and the chi^2 gradients."""
import numpy as np
import pytest
import torch

import synth
from parity import rel

pytestmark = pytest.mark.gpu




@pytest.fixture(scope="module")
def hwp_obs():
    nd, ns = 6, 20000
    o = synth.Observation(64, synth.satellite_scan(ns, t0=40.0), synth.hex_focal_plane(nd))
    o.hwp = synth.hwp_angle(ns, t0=40.0, omega0=0.2)
    return o


@pytest.mark.parametrize("mode", ["cache_f64", "on_the_fly", "cache_mixed", "cache_f32"])
@pytest.mark.parametrize("offsets", [False, True])
def test_hwp_weights_match_oracle(fx, dev, orc, hwp_obs, mode, offsets):
    o = hwp_obs
    delta = np.radians(np.linspace(-1.5, 2.0, o.ndet)) if offsets else None
    opix, oc, os_, _ = orc.pointing(o.nside, o.q_bore, o.q_det, psi_offset=delta, hwp=o.hwp)
    o.psi_offset = delta
    P = fx.Pointing.from_observations([o], mode=mode, device=dev)
    o.psi_offset = None
    pix, c, s = P.expand(torch.float64)
    assert np.array_equal(pix.cpu().numpy(), opix.ravel())
    ok = opix.ravel() >= 0
    tol = 1e-6 if mode == "cache_f32" else 1e-13
    assert np.max(np.abs(c.cpu().numpy()[ok] - oc.ravel()[ok])) < tol
    assert np.max(np.abs(s.cpu().numpy()[ok] - os_.ravel()[ok])) < tol


def test_hwp_operator_matches_oracle(fx, dev, orc, hwp_obs):
    o = hwp_obs
    delta = np.radians(np.linspace(-1.0, 1.0, o.ndet))
    pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det, psi_offset=delta, hwp=o.hwp)
    taps = np.tile(synth.inverse_noise_taps(), (o.ndet, 1))
    on = orc.Noise(taps=taps)
    bj = orc.bj(o.npix, pix, c, s, on)
    x = synth.gaussian_sky(o.nside, synth.rng(7, 5))
    ref = orc.apply_ata(o.npix, pix, c, s, on, bj["valid"], x)
    vt = torch.as_tensor(bj["valid"].astype(np.uint8), device=dev)
    xt = torch.as_tensor(x, device=dev)
    o.psi_offset = delta
    for mode, prec, tol in (("cache_f64", "f64", 1e-12), ("on_the_fly", "f64", 1e-12), ("cache_f32", "f32", 1e-5)):
        P = fx.Pointing.from_observations([o], mode=mode, device=dev)
        N = fx.Noise.banded(P, taps)
        got = fx.ptnp_apply(P, N, xt, vt, precision=prec, acc="f64").cpu().numpy()
        assert rel(got, ref) < tol, mode
        gbj = fx.blockdiag_precond(P, N, 1e-3)
        if mode != "cache_f32":
            assert np.array_equal(gbj["valid"].cpu().numpy(), bj["valid"])
    o.psi_offset = None


def test_hwp_single_detector_recovers_iqu(fx, dev, orc):
    """One detector behind a rotating plate: the noiseless binned map and the PCG map equal the
    input sky on every valid pixel (without the plate most pixels could not be solved)."""
    ns = 40000
    o = synth.Observation(16, synth.satellite_scan(ns), synth.copointed_detectors([0.0]))
    o.hwp = synth.hwp_angle(ns)
    sky = synth.gaussian_sky(o.nside, synth.rng(9, 3))
    P = fx.Pointing.from_observations([o], mode="cache_f64", device=dev)
    N = fx.Noise.white(P, np.array([100.0]))
    d = P.apply(torch.as_tensor(sky, device=dev))
    x, valid, info = fx.mapmaker_cg(P, N, d, maxiter=20, tol=1e-12, precision="f64")
    v = valid.cpu().numpy().astype(bool)
    pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det, hwp=o.hwp)
    assert np.array_equal(v, orc.bj(o.npix, pix, c, s, orc.Noise(sigma2=np.array([100.0])))["valid"])
    assert v.sum() > 1000            # 1476 of 1493 hit pixels with the plate, 178 without it
    assert rel(x.cpu().numpy()[v], sky[v]) < 1e-10


def test_hwp_chi2_gradient_matches_oracle(fx, dev, orc, hwp_obs):
    o = hwp_obs
    g = synth.rng(9, 4)
    delta = np.radians(g.normal(0, 1.0, o.ndet))
    taps = np.tile(synth.inverse_noise_taps(), (o.ndet, 1))
    sky = synth.gaussian_sky(o.nside, g)
    pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det, psi_offset=delta, hwp=o.hwp)
    d = orc.P(pix, c, s, sky) + synth.one_over_f_noise(o.ndet, o.nsamp, g)
    half = delta / 2
    pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det, psi_offset=half, hwp=o.hwp)
    m = sky * 1.01
    chi2, gm, gp = orc.chi2_grad(o.npix, pix, c, s, orc.Noise(taps=taps), m, d, hwp=True)
    o.psi_offset = half
    P = fx.Pointing.from_observations([o], mode="on_the_fly", device=dev)
    o.psi_offset = None
    N = fx.Noise.banded(P, taps)
    c2, gmap, gpsi = fx.chi2_grad(P, N, torch.as_tensor(d.ravel(), device=dev), torch.as_tensor(m, device=dev))
    assert abs(c2.item() - chi2) <= 1e-10 * chi2
    assert rel(gmap.cpu().numpy(), gm) < 1e-9
    assert np.max(np.abs(gpsi.cpu().numpy() - gp)) <= 1e-9 * np.max(np.abs(gp))
