"""Features in combination: template deprojection with a half-wave plate, graph-captured and eager
iterations of the augmented system, long bands on joint maps, chi^2 gradients of a joint map, and
the TOD-ready event with templates. Each is checked against an independent route to the same
quantity (the FP64 solve, the eager solve, the sum over observations)."""
import numpy as np
import pytest
import torch

import synth
from parity import rel
from oracle import templates as ot

pytestmark = pytest.mark.gpu




def demono(m, v):
    m = m[v].copy()
    m[:, 0] -= m[:, 0].mean()
    return m


def tod(obs, seed, drift=100.0):
    g = synth.rng(60, seed)
    return np.concatenate([(synth.one_over_f_noise(o.ndet, o.nsamp, g)
                            + g.normal(size=(o.ndet, 2)) * drift @ ot.legendre_templates(o.nsamp, 1).T).ravel()
                           for o in obs]).astype(np.float32)


def test_templates_with_a_half_wave_plate(fx, dev):
    """Mixed (augmented inner system) and FP64 deprojected solves agree with a rotating plate, in
    the image of the operator. A plate makes pixels crossed by one detector solvable, and with
    offset templates their I trades against that detector's offset: near-null directions that
    FP32 inner iterations cannot resolve, so the maps are compared through A, not directly."""
    obs = [synth.Observation(8, synth.satellite_scan(ns, t0=7.0 * i), synth.hex_focal_plane(nd),
                             hwp=synth.hwp_angle(ns, t0=7.0 * i)) for i, (nd, ns) in enumerate([(4, 9000), (3, 6000)])]
    P = fx.Pointing.from_observations(obs, mode="cache_mixed", device=dev)
    assert P.has_hwp
    N = fx.Noise.banded(P, np.tile(synth.inverse_noise_taps(), (7, 1)))
    T = fx.Templates(P, N, 1)
    d = torch.as_tensor(tod(obs, 0), device=dev)
    x64, v64, i64 = fx.mapmaker_cg(P, N, d, maxiter=500, tol=1e-10, precision="f64", templates=T)
    x32, v32, i32 = fx.mapmaker_cg(P, N, d, maxiter=500, tol=1e-10, precision="f32", templates=T)
    assert i64.converged and i32.converged
    assert np.array_equal(v64.cpu().numpy(), v32.cpu().numpy())
    assert i32.true_rel_res <= 1e-10
    vm = v64.to(torch.uint8)
    ax = fx.ptfp_apply(T, x64, vm, precision="f64", acc="f64")
    ad = fx.ptfp_apply(T, x32 - x64, vm, precision="f64", acc="f64")
    assert float(torch.linalg.norm(ad) / torch.linalg.norm(ax)) < 1e-9


def test_augmented_iterations_graph_equals_eager(fx, dev):
    o = synth.Observation(16, synth.satellite_scan(20000, t0=2.0), synth.hex_focal_plane(6))
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    N = fx.Noise.banded(P, np.tile(synth.inverse_noise_taps(), (6, 1)))
    T = fx.Templates(P, N, 2)
    d = torch.as_tensor(tod([o], 1), device=dev)
    kw = dict(maxiter=30, tol=0.0, precision="f32", acc="f64", inner_tol=0.0, max_outer=1, true_residual=False,
              templates=T)
    xg, vg, _ = fx.mapmaker_cg(P, N, d, use_graph=True, check_every=10, **kw)
    xe, ve, _ = fx.mapmaker_cg(P, N, d, use_graph=False, check_every=7, **kw)
    assert torch.equal(vg, ve)
    # same arithmetic but for the order of the L2 reductions, over 30 iterations of the FP32 operator
    assert rel(xg, xe) < 1e-8


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_long_band_on_joint_maps_is_the_sum_over_observations(fx, dev, prec):
    shapes = [(8, 3, 7000), (8, 2, 12000), (16, 2, 5000)]
    obs = [synth.Observation(n, synth.satellite_scan(ns, t0=5.0 * i), synth.hex_focal_plane(nd), map_id=m)
           for i, ((n, nd, ns), m) in enumerate(zip(shapes, [4, 4, 9]))]
    taps = np.tile(synth.inverse_noise_taps(500), (7, 1))
    P = fx.Pointing.from_observations(obs, mode="cache_f64", device=dev)
    N = fx.Noise.banded(P, taps)
    npix8, npix16 = obs[0].npix, obs[2].npix
    assert P.npix_total == npix8 + npix16
    x = np.concatenate([synth.gaussian_sky(8, synth.rng(61, 0)), synth.gaussian_sky(16, synth.rng(61, 1))])
    got = fx.ptnp_apply(P, N, torch.as_tensor(x, device=dev), None, precision=prec, acc="f64").cpu().numpy()
    ref = np.zeros_like(x)
    offs = [0, 0, npix8]
    rows = [0, 3, 5]
    for o, off, r0 in zip(obs, offs, rows):
        Pi = fx.Pointing.from_observations([synth.Observation(o.nside, o.q_bore, o.q_det)], mode="cache_f64",
                                           device=dev)
        Ni = fx.Noise.banded(Pi, taps[r0:r0 + o.ndet])
        ref[off:off + o.npix] += fx.ptnp_apply(Pi, Ni, torch.as_tensor(x[off:off + o.npix], device=dev), None,
                                               precision=prec, acc="f64").cpu().numpy()
    assert rel(got, ref) < (1e-12 if prec == "f64" else 1e-6)


def test_chi2_gradient_of_a_joint_map_is_the_sum_over_observations(fx, dev):
    shapes = [(8, 3, 6000), (8, 4, 5000)]
    obs = [synth.Observation(n, synth.satellite_scan(ns, t0=3.0 * i), synth.hex_focal_plane(nd), map_id=2)
           for i, (n, nd, ns) in enumerate(shapes)]
    taps = np.tile(synth.inverse_noise_taps(), (7, 1))
    P = fx.Pointing.from_observations(obs, mode="cache_f64", device=dev)
    N = fx.Noise.banded(P, taps)
    m = torch.as_tensor(synth.gaussian_sky(8, synth.rng(62, 0)), device=dev)
    d = torch.as_tensor(tod(obs, 2), device=dev)
    c2, gm, gp = fx.chi2_grad(P, N, d, m)
    c2r, gmr, gpr = 0.0, torch.zeros_like(m), []
    t0 = 0
    for o, r0 in zip(obs, [0, 3]):
        Pi = fx.Pointing.from_observations([synth.Observation(o.nside, o.q_bore, o.q_det)], mode="cache_f64",
                                           device=dev)
        Ni = fx.Noise.banded(Pi, taps[r0:r0 + o.ndet])
        ci, gi, pi = fx.chi2_grad(Pi, Ni, d[t0:t0 + o.ndet * o.nsamp], m)
        c2r += float(ci.sum())
        gmr += gi
        gpr.append(pi)
        t0 += o.ndet * o.nsamp
    assert abs(float(c2.sum()) - c2r) < 1e-10 * abs(c2r)
    assert rel(gm, gmr) < 1e-12
    assert rel(gp, torch.cat(gpr)) < 1e-12


def test_d_ready_with_templates(fx, dev):
    o = synth.Observation(16, synth.satellite_scan(15000, t0=4.0), synth.hex_focal_plane(5))
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    N = fx.Noise.banded(P, np.tile(synth.inverse_noise_taps(), (5, 1)))
    T = fx.Templates(P, N, 1)
    d_h = torch.as_tensor(tod([o], 3)).pin_memory()
    xr, vr, _ = fx.mapmaker_cg(P, N, d_h.to(dev), maxiter=40, tol=0.0, precision="f64", templates=T)
    d = torch.zeros(P.nsamp_total, device=dev)
    torch.cuda.synchronize()
    cs = torch.cuda.Stream(device=dev)
    ev = torch.cuda.Event()
    with torch.cuda.stream(cs):
        d.copy_(d_h, non_blocking=True)
        ev.record(cs)
    x, v, _ = fx.mapmaker_cg(P, N, d, maxiter=40, tol=0.0, precision="f64", templates=T, d_ready=ev)
    assert torch.equal(v, vr)
    assert rel(x, xr) < 1e-12
