"""Edge cases through the C ABI: tiny and odd-length detector streams in one ragged batch (the
cached FP32 operator copies rows on 16-byte boundaries, so odd lengths put row starts anywhere),
an observation whose samples are all invalid, and the largest supported nside."""
import numpy as np
import pytest
import torch

import synth
from parity import elem, rel

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (2, 3), (3, 5), (1, 63), (2, 64), (3, 65), (2, 127), (1, 4095), (2, 4097), (5, 6001)]




@pytest.fixture(scope="module")
def tiny_batch(orc):
    obs = [synth.Observation(8, synth.satellite_scan(ns, t0=37.0 * i), synth.hex_focal_plane(nd))
           for i, (nd, ns) in enumerate(SHAPES)]
    taps = [np.tile(synth.inverse_noise_taps(), (o.ndet, 1)) * (1.0 + 0.1 * i) for i, o in enumerate(obs)]
    x = [synth.gaussian_sky(o.nside, synth.rng(11, i)) for i, o in enumerate(obs)]
    refs = []
    for o, t, xi in zip(obs, taps, x):
        pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det)
        refs.append(orc.apply_ata(o.npix, pix, c, s, orc.Noise(taps=t), None, xi))
    return obs, taps, x, refs


@pytest.mark.parametrize("mode,prec,tol", [("cache_f32", "f32", 2e-6), ("cache_mixed", "f32", 2e-6),
                                           ("cache_f64", "f64", 1e-12), ("on_the_fly", "f64", 1e-12),
                                           ("cache_mixed", "f32x2", 1e-12)])
def test_tiny_and_odd_streams_match_oracle(fx, dev, tiny_batch, mode, prec, tol):
    obs, taps, x, refs = tiny_batch
    P = fx.Pointing.from_observations(obs, mode=mode, device=dev)
    N = fx.Noise.banded(P, np.concatenate(taps))
    xt = torch.as_tensor(np.concatenate(x), device=dev)
    for _ in range(2):   # twice: the second call reuses every workspace
        got = fx.ptnp_apply(P, N, xt, None, precision=prec, acc="f64").cpu().numpy()
        off = 0
        for o, ref in zip(obs, refs):
            assert rel(got[off:off + o.npix], ref) < tol, (o.ndet, o.nsamp)
            off += o.npix


def test_observation_without_valid_samples(fx, dev, orc):
    """All quaternions of one observation are NaN: every sample is invalid, the operator gives
    zeros there, and a solve of that observation alone reports that nothing can be solved."""
    good = synth.Observation(8, synth.satellite_scan(5000), synth.hex_focal_plane(3))
    qb = np.full((3000, 4), np.nan)
    bad = synth.Observation(8, qb, synth.hex_focal_plane(2))
    P = fx.Pointing.from_observations([good, bad], mode="cache_f32", device=dev)
    assert P.n_invalid == 2 * 3000
    pix, _, _ = P.expand()
    assert np.all(pix.cpu().numpy()[3 * 5000:] == -1)
    N = fx.Noise.white(P, np.full(5, 100.0))
    x = torch.randn(P.npix_total, 3, device=dev, dtype=torch.float64)
    y = fx.ptnp_apply(P, N, x, None, precision="f32", acc="f64")
    assert torch.all(y[good.npix:] == 0)
    Pb = fx.Pointing.from_observations([bad], mode="cache_f32", device=dev)
    Nb = fx.Noise.white(Pb, np.full(2, 100.0))
    with pytest.raises(fx.FuraxError) as e:
        fx.mapmaker_cg(Pb, Nb, torch.zeros(Pb.nsamp_total, device=dev), maxiter=5, precision="f64")
    assert e.value.code == -4


@pytest.mark.parametrize("mode", ["on_the_fly", "cache_f64", "cache_f32"])
def test_largest_nside_pixels_bit_exact(fx, dev, orc, mode):
    """nside 8192 (805,306,368 pixels, the largest supported): pixels equal the FP64 recipe."""
    o = synth.Observation(8192, synth.satellite_scan(6000, t0=11.0), synth.hex_focal_plane(4))
    opix, oc, os_, _ = orc.pointing(o.nside, o.q_bore, o.q_det)
    P = fx.Pointing.from_observations([o], mode=mode, device=dev)
    pix, c, s = P.expand()
    assert np.array_equal(pix.cpu().numpy(), opix.ravel())
    ok = opix.ravel() >= 0
    tol = 1e-6 if mode == "cache_f32" else 1e-14
    assert np.max(np.abs(c.cpu().numpy()[ok] - oc.ravel()[ok])) < tol


@pytest.mark.parametrize("mode,prec,tol", [("cache_f32", "f32", 137 * 2.0 ** -24), ("on_the_fly", "f64", 1e-13)])
def test_tiny_and_odd_streams_with_hwp(fx, dev, orc, mode, prec, tol):
    """The same ragged shapes with a rotating half-wave plate on every observation."""
    obs = [synth.Observation(8, synth.satellite_scan(ns, t0=5.0 * i), synth.hex_focal_plane(nd),
                             hwp=synth.hwp_angle(ns, t0=5.0 * i)) for i, (nd, ns) in enumerate(SHAPES)]
    taps = np.tile(synth.inverse_noise_taps(), (sum(o.ndet for o in obs), 1))
    P = fx.Pointing.from_observations(obs, mode=mode, device=dev)
    assert P.has_hwp
    N = fx.Noise.banded(P, taps)
    x = [synth.gaussian_sky(o.nside, synth.rng(12, i)) for i, o in enumerate(obs)]
    got = fx.ptnp_apply(P, N, torch.as_tensor(np.concatenate(x), device=dev), None, precision=prec,
                        acc="f64").cpu().numpy()
    off = 0
    for o, xi in zip(obs, x):
        pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det, hwp=o.hwp)
        on = orc.Noise(taps=taps[:o.ndet])
        ref = orc.apply_ata(o.npix, pix, c, s, on, None, xi)
        # per element against |P^T||N^-1||P||x|: in FP32 the weights (rounded once, 2^-24), the map
        # and the 127-term band in FP32 arithmetic bound the error by ~(129 + 8) u
        scale = orc.apply_ata(o.npix, pix, np.abs(c), np.abs(s), orc.Noise(taps=np.abs(taps[:o.ndet])), None,
                              np.abs(xi))
        assert elem(got[off:off + o.npix], ref, scale) < tol, (o.ndet, o.nsamp)
        off += o.npix
