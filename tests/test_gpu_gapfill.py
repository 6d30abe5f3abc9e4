"""Gap filling by constrained Gaussian realisation on the GPU against the FP64 oracle."""
import numpy as np
import pytest
import torch

import synth
from parity import rel
from oracle import gapfill as og

pytestmark = pytest.mark.gpu




# streams of 1 sample, shorter than the band, one tile, several tiles with a ragged tail
SHAPES = [(1, 1), (2, 50), (3, 4096), (2, 9001)]


def make(ntaps, seed):
    obs = [synth.Observation(8, synth.satellite_scan(ns, t0=3.0 * i), synth.hex_focal_plane(nd))
           for i, (nd, ns) in enumerate(SHAPES)]
    g = np.random.default_rng(seed)
    cov = [np.tile(synth.noise_covariance_band(ntaps), (o.ndet, 1)) * (1 + 0.5 * np.arange(o.ndet))[:, None]
           for o in obs]
    n = [synth.band_realization(c, o.nsamp, g) for o, c in zip(obs, cov)]
    d = [synth.band_realization(c, o.nsamp, g) + 5.0 for o, c in zip(obs, cov)]
    valid = []
    for o in obs:
        v = g.random((o.ndet, o.nsamp)) > 0.1
        if o.nsamp > 400:
            v[:, 200:320] = False   # a long gap
        v[:, :2] = False            # gaps at the start of each stream
        valid.append(v)
    return obs, cov, d, n, valid


def cat(xs):
    return np.concatenate([x.ravel() for x in xs])


@pytest.mark.parametrize("ntaps", [64, 300])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-8), (torch.float32, 2e-6)])
@pytest.mark.parametrize("precision", ["f64", "f32x2"])   # f32x2: double-FP32 band products (64 taps)
def test_gapfill_matches_oracle(fx, dev, ntaps, dtype, tol, precision):
    obs, cov, d, n, valid = make(ntaps, ntaps)
    if dtype == torch.float32:
        d = [x.astype(np.float32).astype(np.float64) for x in d]
        n = [x.astype(np.float32).astype(np.float64) for x in n]
    P = fx.Pointing.from_observations(obs, mode="cache_f32", device=dev)
    N = fx.Noise.banded(P, np.concatenate(cov))
    dt = torch.as_tensor(cat(d), device=dev, dtype=dtype)
    out, iters, ok = fx.gapfill(N, dt, torch.as_tensor(cat(valid), device=dev), torch.as_tensor(cat(n), device=dev,
                                                                                               dtype=dtype),
                                maxiter=2000, tol=1e-12, precision=precision)
    assert ok
    got = out.double().cpu().numpy()
    off = 0
    for o, c, di, ni, vi in zip(obs, cov, d, n, valid):
        m = o.ndet * o.nsamp
        ref, _ = og.gapfill(c, di, vi, ni, tol=1e-13)
        gi = got[off:off + m].reshape(o.ndet, o.nsamp)
        assert np.array_equal(gi[vi], di[vi])                           # observed samples untouched
        if (~vi).any():
            assert rel(gi[~vi], ref[~vi]) < tol, (o.ndet, o.nsamp)
        off += m


def test_gapfill_special_cases(fx, dev):
    obs, cov, d, n, valid = make(64, 3)
    P = fx.Pointing.from_observations(obs, mode="cache_f32", device=dev)
    N = fx.Noise.banded(P, np.concatenate(cov))
    dt, nt = torch.as_tensor(cat(d), device=dev), torch.as_tensor(cat(n), device=dev)
    ones = torch.ones(P.nsamp_total, dtype=torch.uint8, device=dev)
    out, _, ok = fx.gapfill(N, dt, ones, nt)
    assert ok and torch.equal(out, dt)                                   # nothing to fill
    out, iters, ok = fx.gapfill(N, dt, torch.zeros_like(ones), nt)
    assert ok and torch.equal(out, nt) and max(iters) == 0              # nothing observed
    out, iters, ok = fx.gapfill(N, nt, torch.as_tensor(cat(valid), device=dev), nt)
    assert ok and torch.equal(out, nt) and max(iters) == 0              # data equal to the realisation
    out, iters, ok = fx.gapfill(N, dt, torch.as_tensor(cat(valid), device=dev), nt, maxiter=3)
    assert not ok and max(iters) == 3                                   # stopped at the cap, still written
    assert torch.equal(out[ones.bool() & torch.as_tensor(cat(valid), device=dev)],
                       dt[torch.as_tensor(cat(valid), device=dev)])


def test_gapfill_full_scale_sampled(fx, dev):
    """64 detectors x 2^20 samples with 10 % of the samples in gaps (random and 2000-sample
    stretches), 300-tap covariance (overlap-save product): detectors 0 and 63 against the oracle."""
    ns, nd = 1 << 20, 64
    o = synth.Observation(256, synth.satellite_scan(ns), synth.hex_focal_plane(nd))
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    c = synth.noise_covariance_band(300)
    N = fx.Noise.banded(P, np.tile(c, (nd, 1)))
    g = np.random.default_rng(7)
    rows = [0, nd - 1]
    d = np.zeros((nd, ns), np.float32)
    n = np.zeros((nd, ns), np.float32)
    for r in rows:
        d[r] = synth.band_realization(c, ns, g)[0] + 2.0
        n[r] = synth.band_realization(c, ns, g)[0]
    valid = g.random((nd, ns)) > 0.08
    for start in range(5000, ns, 100000):
        valid[:, start:start + 2000] = False
    out, iters, ok = fx.gapfill(N, torch.as_tensor(d.ravel(), device=dev), torch.as_tensor(valid.ravel(), device=dev),
                                torch.as_tensor(n.ravel(), device=dev), maxiter=3000, tol=1e-10)
    assert ok
    got = out.cpu().numpy().reshape(nd, ns)
    for r in rows:
        ref, _ = og.gapfill(c[None, :], d[r:r + 1].astype(np.float64), valid[r:r + 1], n[r:r + 1].astype(np.float64),
                            tol=1e-11)
        gap = ~valid[r]
        assert np.array_equal(got[r][valid[r]], d[r][valid[r]])
        assert rel(got[r][gap], ref[0][gap]) < 1e-5


@pytest.mark.parametrize("ntaps", [64, 300])
def test_gapfill_fp32_operator(fx, dev, ntaps):
    """precision f32: N applied in FP32, CG vectors and scalars in FP64; the filled values follow
    the oracle to the FP32 band product's accuracy."""
    obs, cov, d, n, valid = make(ntaps, 100 + ntaps)
    P = fx.Pointing.from_observations(obs, mode="cache_f32", device=dev)
    N = fx.Noise.banded(P, np.concatenate(cov))
    out, iters, ok = fx.gapfill(N, torch.as_tensor(cat(d), device=dev), torch.as_tensor(cat(valid), device=dev),
                                torch.as_tensor(cat(n), device=dev), maxiter=2000, tol=1e-8, precision="f32")
    assert ok
    got = out.cpu().numpy()
    off = 0
    for o, c, di, ni, vi in zip(obs, cov, d, n, valid):
        m = o.ndet * o.nsamp
        ref, _ = og.gapfill(c, di, vi, ni, tol=1e-13)
        gi = got[off:off + m].reshape(o.ndet, o.nsamp)
        assert np.array_equal(gi[vi], di[vi])
        if (~vi).any():
            assert rel(gi[~vi], ref[~vi]) < 1e-5, (o.ndet, o.nsamp)
        off += m


def test_gapfill_rejects_a_white_handle(fx, dev):
    o = synth.Observation(8, synth.satellite_scan(100), synth.hex_focal_plane(2))
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    W = fx.Noise.white(P, np.ones(2))
    x = torch.zeros(P.nsamp_total, device=dev)
    with pytest.raises(ValueError):
        fx.gapfill(W, x, torch.ones_like(x, dtype=torch.uint8), x)
    out = torch.empty_like(x)
    with pytest.raises(fx.FuraxError) as e:
        fx._native.furax_gapfill(W.handle, 2, x, torch.ones_like(x, dtype=torch.uint8), x, out)
    assert e.value.code == -1


def test_workspaces_are_reused_across_calls_and_precisions(fx, dev):
    """The handle keeps the gap-filling workspaces: a repeated call reproduces the first bit for bit,
    and switching precision on the same handle (which adds the FP64 band-product vector) changes
    nothing for the FP32 call that follows."""
    obs, cov, d, n, valid = make(64, 5)
    P = fx.Pointing.from_observations(obs, mode="cache_f32", device=dev)
    N = fx.Noise.banded(P, np.concatenate(cov))
    dt = torch.as_tensor(cat(d), device=dev)
    vt = torch.as_tensor(cat(valid), device=dev)
    nt = torch.as_tensor(cat(n), device=dev)
    kw = dict(maxiter=2000, tol=1e-10)
    a, ia, oka = fx.gapfill(N, dt, vt, nt, precision="f32", **kw)
    b, ib, okb = fx.gapfill(N, dt, vt, nt, precision="f32", **kw)
    c, ic, okc = fx.gapfill(N, dt, vt, nt, precision="f64", **kw)
    e, ie, oke = fx.gapfill(N, dt, vt, nt, precision="f32", **kw)
    assert oka and okb and okc and oke
    assert torch.equal(a, b) and torch.equal(a, e)
    assert list(ia) == list(ib) == list(ie)
    assert rel(a.cpu().numpy(), c.cpu().numpy()) < 1e-6
