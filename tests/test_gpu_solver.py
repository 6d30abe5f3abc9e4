"""GPU map-making vs the FP64 oracle: binned map, FP64 PCG, mixed-precision PCG with defect
correction to a true residual of 1e-8, per-observation batched solves, graph vs eager."""
import numpy as np
import pytest
import torch

import synth
from parity import rel

pytestmark = pytest.mark.gpu




@pytest.fixture(scope="module")
def c1(orc):
    obs, sky, noise, sigma2 = synth.config1()
    pix, c, s, _ = orc.pointing(obs.nside, obs.q_bore, obs.q_det)
    d = orc.P(pix, c, s, sky) + noise
    nz = orc.Noise(sigma2=sigma2)
    bj = orc.bj(obs.npix, pix, c, s, nz)
    b = orc.rhs(obs.npix, pix, c, s, nz, bj["valid"], d)
    return obs, sky, d, sigma2, pix, c, s, nz, bj, b


def test_c1_binned_and_pcg_fp64(fx, dev, orc, c1):
    obs, sky, d, sigma2, pix, c, s, nz, bj, b = c1
    P = fx.Pointing.from_observations([obs], mode="cache_f64", device=dev)
    N = fx.Noise.white(P, sigma2)
    dt = torch.as_tensor(d.ravel(), device=dev)
    v = bj["valid"]
    xb, valid, info = fx.mapmaker_cg(P, N, dt, binned_only=True)
    assert np.array_equal(valid.cpu().numpy(), v)
    ref_binned = orc.binned_map(bj, b)
    assert rel(xb.cpu().numpy()[v], ref_binned[v]) < 1e-10
    x, valid, info = fx.mapmaker_cg(P, N, dt, maxiter=30, tol=1e-8, precision="f64")
    ox, it, hist = orc.pcg(obs.npix, pix, c, s, nz, v, bj["inv"], b, 30, 1e-8)
    assert info.converged and info.iters == it == 1   # white noise: one step to the binned map
    assert rel(x.cpu().numpy()[v], ox[v]) < 1e-10
    assert np.all(x.cpu().numpy()[~v] == 0)
    assert info.true_rel_res < 1e-12
    assert info.n_valid == v.sum()


@pytest.fixture(scope="module")
def banded(orc):
    """Reduced config-2 geometry: nside 64, 32 hex detectors x 16384 samples, 1/f noise."""
    o = synth.Observation(64, synth.satellite_scan(16384, t0=50.0), synth.hex_focal_plane(32))
    pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det)
    sky = synth.gaussian_sky(o.nside, synth.rng(2, 0))
    d = (orc.P(pix, c, s, sky) + synth.one_over_f_noise(32, 16384, synth.rng(2, 1))).astype(np.float32)
    taps = np.tile(synth.inverse_noise_taps(), (32, 1))
    nz = orc.Noise(taps=taps)
    bj = orc.bj(o.npix, pix, c, s, nz)
    b = orc.rhs(o.npix, pix, c, s, nz, bj["valid"], d.astype(np.float64))
    return o, sky, d, taps, pix, c, s, nz, bj, b


def test_banded_pcg_fp64_matches_oracle_iterates(fx, dev, orc, banded):
    o, sky, d, taps, pix, c, s, nz, bj, b = banded
    P = fx.Pointing.from_observations([o], mode="cache_f64", device=dev)
    N = fx.Noise.banded(P, taps)
    v = bj["valid"]
    dt = torch.as_tensor(d.ravel(), device=dev)
    for k in (1, 5, 20):
        x, valid, info = fx.mapmaker_cg(P, N, dt, maxiter=k, tol=0.0, precision="f64", check_every=5)
        ox, it, hist = orc.pcg(o.npix, pix, c, s, nz, v, bj["inv"], b, k, 0.0)
        assert info.iters == it == k
        assert rel(x.cpu().numpy()[v], ox[v]) < 1e-9, k
        np.testing.assert_allclose(info.history[1:], hist[1:], rtol=1e-7)


def test_banded_pcg_converges_fp64_and_mixed(fx, dev, orc, banded):
    o, sky, d, taps, pix, c, s, nz, bj, b = banded
    v = bj["valid"]
    ox, it, hist = orc.pcg(o.npix, pix, c, s, nz, v, bj["inv"], b, 2000, 1e-12)
    dt = torch.as_tensor(d.ravel(), device=dev)
    P64 = fx.Pointing.from_observations([o], mode="cache_f64", device=dev)
    x64, _, i64 = fx.mapmaker_cg(P64, fx.Noise.banded(P64, taps), dt, maxiter=2000, tol=1e-8, precision="f64")
    assert i64.converged and i64.true_rel_res <= 1.5e-8
    P32 = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    for acc in ("f32", "f32_kahan", "f64"):
        x32, _, i32 = fx.mapmaker_cg(P32, fx.Noise.banded(P32, taps), dt, maxiter=2000, tol=1e-8, precision="f32",
                                     acc=acc, inner_tol=1e-5)
        assert i32.converged, (acc, i32)
        assert i32.true_rel_res <= 1e-8
        assert i32.outer >= 1
        # the FP32 cache holds rounded weights: this solve converges for the operator with those
        # weights, which differs from the FP64 one by the rounding (~1e-7)
        assert rel(x32.cpu().numpy()[v], ox[v]) < 1e-5, acc
    # the mixed cache keeps hi + lo weights: inner FP32 operator, outer FP64-accurate operator,
    # so the mixed solve reaches the FP64 system's solution at the FP64 solve's tolerance
    PM = fx.Pointing.from_observations([o], mode="cache_mixed", device=dev)
    xm, _, im = fx.mapmaker_cg(PM, fx.Noise.banded(PM, taps), dt, maxiter=2000, tol=1e-8, precision="f32",
                               acc="f32", inner_tol=1e-5)
    assert im.converged and im.true_rel_res <= 1e-8
    assert rel(xm.cpu().numpy()[v], ox[v]) < 1e-6
    assert rel(xm.cpu().numpy()[v], x64.cpu().numpy()[v]) < 1e-6
    assert rel(x64.cpu().numpy()[v], ox[v]) < 1e-6


def test_noiseless_recovery_mixed(fx, dev, orc, banded):
    o, sky, d, taps, pix, c, s, nz, bj, b = banded
    v = bj["valid"]
    m = sky.copy()
    m[~v] = 0.0
    P = fx.Pointing.from_observations([o], mode="cache_f64", device=dev)
    N = fx.Noise.banded(P, taps)
    dn = P.apply(torch.as_tensor(m, device=dev), dtype=torch.float64)
    # solved to 1e-13: the per-component error of Q and U (100 times smaller than I) then stays
    # below 1e-10 of their own scale
    x, valid, info = fx.mapmaker_cg(P, N, dn, maxiter=3000, tol=1e-13, precision="f64")
    assert rel(x.cpu().numpy()[v], m[v]) < 1e-10


def test_graph_and_eager_identical(fx, dev, banded):
    o, sky, d, taps, *_ = banded
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    N = fx.Noise.banded(P, taps)
    dt = torch.as_tensor(d.ravel(), device=dev)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        xg, _, ig = fx.mapmaker_cg(P, N, dt, maxiter=30, tol=0.0, precision="f64", use_graph=True, check_every=10)
        xe, _, ie = fx.mapmaker_cg(P, N, dt, maxiter=30, tol=0.0, precision="f64", use_graph=False, check_every=7)
    s.synchronize()
    assert ig.iters == ie.iters == 30
    # dots are reduced in a fixed order; the scatter's FP64 atomics are not, so the two runs
    # differ only by that rounding order, amplified over 30 iterations
    assert (torch.linalg.norm(xg - xe) / torch.linalg.norm(xe)).item() < 1e-9


def test_batched_observations_solved_independently(fx, dev, orc):
    """Ragged batch (per-observation nside, ndet, nsamp): each observation's PCG equals the oracle's."""
    shapes = [(16, 4, 6000), (32, 9, 4097), (16, 12, 9000), (64, 5, 12000)]
    obs = [synth.Observation(ns, synth.satellite_scan(n, t0=300.0 * i), synth.hex_focal_plane(nd))
           for i, (ns, nd, n) in enumerate(shapes)]
    taps_all, d_all, refs = [], [], []
    for i, o in enumerate(obs):
        pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det)
        taps = np.tile(synth.inverse_noise_taps(), (o.ndet, 1))
        nz = orc.Noise(taps=taps)
        sky = synth.gaussian_sky(o.nside, synth.rng(4, 10 + i))
        d = orc.P(pix, c, s, sky) + synth.one_over_f_noise(o.ndet, o.nsamp, synth.rng(4, 20 + i))
        bj = orc.bj(o.npix, pix, c, s, nz)
        b = orc.rhs(o.npix, pix, c, s, nz, bj["valid"], d)
        ox, it, _ = orc.pcg(o.npix, pix, c, s, nz, bj["valid"], bj["inv"], b, 15, 0.0)
        refs.append((ox, bj["valid"]))
        taps_all.append(taps)
        d_all.append(d.ravel())
    P = fx.Pointing.from_observations(obs, mode="cache_f64", device=dev)
    N = fx.Noise.banded(P, np.concatenate(taps_all))
    x, valid, info = fx.mapmaker_cg(P, N, torch.as_tensor(np.concatenate(d_all), device=dev), maxiter=15, tol=0.0,
                                    precision="f64")
    x = x.cpu().numpy()
    valid = valid.cpu().numpy()
    off = 0
    for o, (ox, v) in zip(obs, refs):
        assert np.array_equal(valid[off:off + o.npix], v)
        assert rel(x[off:off + o.npix][v], ox[v]) < 1e-9
        off += o.npix


def test_maxiter_cap_reports_not_converged(fx, dev, banded):
    o, sky, d, taps, *_ = banded
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    x, _, info = fx.mapmaker_cg(P, fx.Noise.banded(P, taps), torch.as_tensor(d.ravel(), device=dev), maxiter=3,
                                tol=1e-12, precision="f64")
    assert not info.converged and info.iters == 3


def test_pcg_converges_with_precession_repeats(fx, dev, orc):
    """A scan longer than one precession period: with positive definite preconditioner blocks,
    block-Jacobi PCG keeps its fast convergence (spectrum of M^-1 A within the band's symbol
    ratio), FP64 and mixed precision reach the same map, and both match the oracle."""
    o = synth.Observation(256, synth.satellite_scan(160000), synth.hex_focal_plane(4))
    pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det)
    taps = np.tile(synth.inverse_noise_taps(), (4, 1))
    nz = orc.Noise(taps=taps)
    d = (orc.P(pix, c, s, synth.gaussian_sky(o.nside, synth.rng(2, 0)))
         + synth.one_over_f_noise(4, 160000, synth.rng(2, 1))).astype(np.float32)
    bj = orc.bj(o.npix, pix, c, s, nz, 1e-2)
    v = bj["valid"]
    b = orc.rhs(o.npix, pix, c, s, nz, v, d.astype(np.float64))
    ox, it, _ = orc.pcg(o.npix, pix, c, s, nz, v, bj["inv"], b, 200, 1e-12)
    assert it < 60
    dt = torch.as_tensor(d.ravel(), device=dev)
    P64 = fx.Pointing.from_observations([o], mode="cache_f64", device=dev)
    x64, _, i64 = fx.mapmaker_cg(P64, fx.Noise.banded(P64, taps), dt, maxiter=200, tol=1e-8, precision="f64",
                                 rcond_min=1e-2)
    assert i64.converged and i64.iters < 40 and i64.true_rel_res <= 1.5e-8
    PM = fx.Pointing.from_observations([o], mode="cache_mixed", device=dev)
    xm, _, im = fx.mapmaker_cg(PM, fx.Noise.banded(PM, taps), dt, maxiter=400, tol=1e-8, precision="f32",
                               acc="f32", inner_tol=1e-5, rcond_min=1e-2)
    assert im.converged and im.true_rel_res <= 1e-8
    assert rel(x64.cpu().numpy()[v], ox[v]) < 1e-6
    assert rel(xm.cpu().numpy()[v], ox[v]) < 1e-6


def test_d_ready_event_orders_the_tod_upload(fx, dev):
    """d copied from pinned host memory on another stream, with its event passed as d_ready, gives
    the solve of the same data already on the device (the solver waits only where it reads d)."""
    o = synth.Observation(16, synth.satellite_scan(20000, t0=9.0), synth.hex_focal_plane(8))
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    N = fx.Noise.banded(P, np.tile(synth.inverse_noise_taps(), (8, 1)))
    d_h = torch.randn(P.nsamp_total, generator=torch.Generator().manual_seed(3)).pin_memory()
    xr, vr, _ = fx.mapmaker_cg(P, N, d_h.to(dev), maxiter=30, tol=0.0, precision="f64")
    d = torch.zeros(P.nsamp_total, device=dev)
    torch.cuda.synchronize()
    cs = torch.cuda.Stream(device=dev)
    ev = torch.cuda.Event()
    with torch.cuda.stream(cs):
        d.copy_(d_h, non_blocking=True)
        ev.record(cs)
    x, v, _ = fx.mapmaker_cg(P, N, d, maxiter=30, tol=0.0, precision="f64", d_ready=ev)
    assert torch.equal(v, vr)
    assert (torch.linalg.norm(x - xr) / torch.linalg.norm(xr)).item() < 1e-12
