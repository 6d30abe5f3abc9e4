"""Long symmetric bands (65..2048 taps): N^-1 by overlap-save (SymmetricBandToeplitzOperator of
Table 2, one of whose evaluations is overlap-save) and the map-making operators built on it,
against the oracle's direct sum."""
import numpy as np
import pytest
import torch

import synth
from parity import rel
from oracle import templates as ot

pytestmark = pytest.mark.gpu




# streams of one sample, shorter than the band, one block, an odd and an even number of blocks
SHAPES = [(1, 1), (2, 700), (3, 6000), (2, 20000), (1, 37000)]


def batch(nside=8):
    return [synth.Observation(nside, synth.satellite_scan(ns, t0=17.0 * i), synth.hex_focal_plane(nd))
            for i, (nd, ns) in enumerate(SHAPES)]


@pytest.mark.parametrize("ntaps", [65, 300, 2048])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
def test_overlap_save_matches_direct_band(fx, dev, orc, ntaps, dtype, tol):
    obs = batch()
    P = fx.Pointing.from_observations(obs, mode="cache_f32", device=dev)
    taps = [np.tile(synth.inverse_noise_taps(ntaps), (o.ndet, 1)) * (1 + 0.3 * np.arange(o.ndet))[:, None]
            for o in obs]
    N = fx.Noise.banded(P, np.concatenate(taps))
    g = np.random.default_rng(ntaps)
    x = np.concatenate([g.normal(size=o.ndet * o.nsamp) for o in obs])
    if dtype == torch.float32:
        x = x.astype(np.float32).astype(np.float64)
    y = N.inv_apply(torch.as_tensor(x, device=dev, dtype=dtype)).double().cpu().numpy()
    off = 0
    for o, t in zip(obs, taps):
        n = o.ndet * o.nsamp
        ref = orc.ninv_band(t, x[off:off + n].reshape(o.ndet, o.nsamp)).ravel()
        assert rel(y[off:off + n], ref) < tol, (o.ndet, o.nsamp)
        off += n


@pytest.fixture(scope="module")
def problem(orc):
    o = synth.Observation(8, synth.satellite_scan(30000, t0=3.0), synth.hex_focal_plane(6))
    pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det)
    taps = np.tile(synth.inverse_noise_taps(1024), (6, 1)) * np.linspace(0.9, 1.1, 6)[:, None]
    return o, pix, c, s, taps


@pytest.mark.parametrize("mode,prec,tol", [("cache_f64", "f64", 1e-12), ("on_the_fly", "f32x2", 1e-12),
                                           ("cache_f32", "f32", 1e-5)])
def test_normal_operator_and_rhs_with_a_long_band(fx, dev, orc, problem, mode, prec, tol):
    o, pix, c, s, taps = problem
    P = fx.Pointing.from_observations([o], mode=mode, device=dev)
    N = fx.Noise.banded(P, taps)
    on = orc.Noise(taps=taps)
    valid = orc.bj(o.npix, pix, c, s, on)["valid"]
    x = synth.gaussian_sky(o.nside, synth.rng(50, 0))
    ref = orc.apply_ata(o.npix, pix, c, s, on, valid, x)
    vt = torch.as_tensor(valid.astype(np.uint8), device=dev)
    got = fx.ptnp_apply(P, N, torch.as_tensor(x, device=dev), vt, precision=prec, acc="f32").cpu().numpy()
    assert rel(got, ref) < tol
    d = synth.one_over_f_noise(6, 30000, synth.rng(50, 1)).astype(np.float32)
    rref = orc.rhs(o.npix, pix, c, s, on, valid, d.astype(np.float64))
    b = fx.rhs(P, N, torch.as_tensor(d.ravel(), device=dev), vt).cpu().numpy()
    # the right-hand side is FP64 whatever the pointing cache; the FP32 cache's weights carry ~1e-7
    assert rel(b, rref) < (2e-6 if mode == "cache_f32" else 1e-12)


@pytest.mark.parametrize("precision,mode,tol", [("f64", "cache_f64", 1e-9), ("f32", "cache_mixed", 1e-7)])
def test_solve_with_a_long_band_matches_oracle(fx, dev, orc, problem, precision, mode, tol):
    o, pix, c, s, taps = problem
    on = orc.Noise(taps=taps)
    g = synth.rng(51, 0)
    d = (orc.P(pix, c, s, synth.gaussian_sky(o.nside, g)) + synth.one_over_f_noise(6, 30000, g)).astype(np.float32)
    bjd = orc.bj(o.npix, pix, c, s, on)
    b = orc.rhs(o.npix, pix, c, s, on, bjd["valid"], d.astype(np.float64))
    xo, _, hist = orc.pcg(o.npix, pix, c, s, on, bjd["valid"], bjd["inv"], b, 300, 1e-12)
    assert hist[-1] <= 1e-12
    P = fx.Pointing.from_observations([o], mode=mode, device=dev)
    N = fx.Noise.banded(P, taps)
    x, valid, info = fx.mapmaker_cg(P, N, torch.as_tensor(d.ravel(), device=dev), maxiter=300, tol=1e-11,
                                    precision=precision)
    assert info.converged and info.true_rel_res <= 1e-11
    v = valid.cpu().numpy()
    assert np.array_equal(v, bjd["valid"])
    assert rel(x.cpu().numpy()[v], xo[v]) < tol


def test_templates_with_a_long_band(fx, dev, orc, problem):
    o, pix, c, s, taps = problem
    P = fx.Pointing.from_observations([o], mode="cache_f64", device=dev)
    N = fx.Noise.banded(P, taps)
    T = fx.Templates(P, N, 1)
    on = orc.Noise(taps=taps)
    assert rel(T.gram().cpu().numpy(), ot.gram(on, 6, 30000, 1)) < 1e-12
    x = synth.gaussian_sky(o.nside, synth.rng(52, 0))
    ref = ot.ptfp_apply(o.npix, pix, c, s, on, 1, None, x)
    got = fx.ptfp_apply(T, torch.as_tensor(x, device=dev), None, precision="f64", acc="f64").cpu().numpy()
    assert rel(got, ref) < 1e-11


def test_long_band_limits(fx, dev):
    o = synth.Observation(8, synth.satellite_scan(500), synth.hex_focal_plane(2))
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    with pytest.raises(fx.FuraxError) as e:
        fx.Noise.banded(P, np.tile(synth.inverse_noise_taps(2049), (2, 1)))
    assert e.value.code == -1
    N = fx.Noise.banded(P, np.tile(synth.inverse_noise_taps(100), (2, 1)))
    d = torch.zeros(P.nsamp_total, device=dev)
    m = torch.zeros(P.npix_total, 3, dtype=torch.float64, device=dev)
    with pytest.raises(fx.FuraxError) as e:
        fx.chi2_grad(P, N, d, m)
    assert e.value.code == -1
