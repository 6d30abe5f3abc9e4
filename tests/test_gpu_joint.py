"""Joint maps: observations sharing a map_id are solved into one map ("Algebraic reductions":
P^T N^-1 P = sum_i P_i^T N_i^-1 P_i over the observations of the map)."""
import numpy as np
import pytest
import torch

import synth
from parity import rel

pytestmark = pytest.mark.gpu




def obs_list(shapes, ids):
    return [synth.Observation(nside, synth.satellite_scan(ns, t0=211.0 * i), synth.hex_focal_plane(nd), map_id=m)
            for i, ((nside, nd, ns), m) in enumerate(zip(shapes, ids))]


# three observations onto map 5 (nside 8, ragged lengths), two onto map 9 (nside 16), one alone
SHAPES = [(8, 4, 5000), (16, 3, 4096), (8, 6, 9001), (16, 5, 300), (8, 2, 64), (4, 3, 7000)]
IDS = [5, 9, 5, 9, 5, 7]


def map_layout(obs):
    """First-appearance order of the maps: {map_id: (offset, npix)}."""
    out, off = {}, 0
    for o in obs:
        if o.map_id not in out:
            out[o.map_id] = (off, o.npix)
            off += o.npix
    return out


@pytest.mark.parametrize("prec,acc,mode,tol", [("f64", "f64", "cache_f64", 1e-13), ("f32", "f64", "cache_f32", 1e-12),
                                               ("f32x2", "f64", "cache_mixed", 1e-13)])
def test_joint_operator_is_the_sum_over_its_observations(fx, dev, prec, acc, mode, tol):
    obs = obs_list(SHAPES, IDS)
    lay = map_layout(obs)
    taps = [np.tile(synth.inverse_noise_taps(), (o.ndet, 1)) * (1 + 0.1 * i) for i, o in enumerate(obs)]
    P = fx.Pointing.from_observations(obs, mode=mode, device=dev)
    assert P.npix_total == sum(n for _, n in lay.values())
    N = fx.Noise.banded(P, np.concatenate(taps))
    x = np.concatenate([synth.gaussian_sky(obs[[o.map_id for o in obs].index(m)].nside, synth.rng(40, k))
                        for k, m in enumerate(lay)])
    got = fx.ptnp_apply(P, N, torch.as_tensor(x, device=dev), None, precision=prec, acc=acc).cpu().numpy()
    ref = np.zeros_like(x)
    for o, t in zip(obs, taps):
        off, npix = lay[o.map_id]
        Pi = fx.Pointing.from_observations([synth.Observation(o.nside, o.q_bore, o.q_det)], mode=mode, device=dev)
        Ni = fx.Noise.banded(Pi, t)
        ref[off:off + npix] += fx.ptnp_apply(Pi, Ni, torch.as_tensor(x[off:off + npix], device=dev), None,
                                             precision=prec, acc=acc).cpu().numpy()
    assert rel(got, ref) < tol
    # P reads the shared map: each observation's TOD equals its own handle's
    tod = P.apply(torch.as_tensor(x, device=dev), dtype=torch.float64).cpu().numpy()
    t0 = 0
    for o in obs:
        off, npix = lay[o.map_id]
        Pi = fx.Pointing.from_observations([synth.Observation(o.nside, o.q_bore, o.q_det)], mode=mode, device=dev)
        ti = Pi.apply(torch.as_tensor(x[off:off + npix], device=dev), dtype=torch.float64).cpu().numpy()
        assert np.array_equal(tod[t0:t0 + o.ndet * o.nsamp], ti)
        t0 += o.ndet * o.nsamp


@pytest.fixture(scope="module")
def joint_case(orc):
    """Three observations of 12000 samples (4, 6, 5 detectors, different scan phases) onto one
    nside-8 map. The oracle sees them as one observation of 15 detectors on that map."""
    shapes = [(8, 4, 12000), (8, 6, 12000), (8, 5, 12000)]
    obs = obs_list(shapes, [3, 3, 3])
    pts = [orc.pointing(o.nside, o.q_bore, o.q_det)[:3] for o in obs]
    pix, c, s = (np.concatenate([p[k] for p in pts]) for k in range(3))
    taps = np.tile(synth.inverse_noise_taps(), (15, 1)) * np.linspace(0.8, 1.2, 15)[:, None]
    g = synth.rng(41, 0)
    d = orc.P(pix, c, s, synth.gaussian_sky(8, g)) + synth.one_over_f_noise(15, 12000, g)
    d = d.astype(np.float32).astype(np.float64)
    on = orc.Noise(taps=taps)
    bjd = orc.bj(obs[0].npix, pix, c, s, on, rcond_min=1e-3)
    b = orc.rhs(obs[0].npix, pix, c, s, on, bjd["valid"], d)
    xo, it, hist = orc.pcg(obs[0].npix, pix, c, s, on, bjd["valid"], bjd["inv"], b, 400, 1e-12)
    return obs, taps, d, bjd, xo


@pytest.mark.parametrize("precision,mode,tol", [("f64", "cache_f64", 1e-9), ("f32", "cache_mixed", 1e-7),
                                                ("f32", "cache_f32", 1e-5)])
def test_joint_solve_matches_oracle(fx, dev, joint_case, precision, mode, tol):
    obs, taps, d, bjd, xo = joint_case
    P = fx.Pointing.from_observations(obs, mode=mode, device=dev)
    assert P.npix_total == obs[0].npix
    N = fx.Noise.banded(P, taps)
    # both sides solve to a relative residual of 1e-12, so that the stopping point does not decide the
    # per-component comparison (Q and U are ~100 times smaller than I)
    x, valid, info = fx.mapmaker_cg(P, N, torch.as_tensor(d.ravel().astype(np.float32), device=dev), maxiter=400,
                                    tol=1e-12, precision=precision)
    assert info.converged
    v = valid.cpu().numpy()
    assert np.array_equal(v, bjd["valid"])
    assert rel(x.cpu().numpy()[v], xo[v]) < tol


def test_maps_of_one_batch_are_independent(fx, dev, orc):
    """A batch holding two joint maps and a lone observation gives, map by map, the solves of
    those observations on their own."""
    obs = obs_list(SHAPES, IDS)
    taps = np.tile(synth.inverse_noise_taps(), (sum(o.ndet for o in obs), 1))
    g = np.random.default_rng(42)
    d = [g.normal(size=o.ndet * o.nsamp) * 30.0 for o in obs]
    P = fx.Pointing.from_observations(obs, mode="cache_f64", device=dev)
    N = fx.Noise.banded(P, taps)
    x, valid, info = fx.mapmaker_cg(P, N, torch.as_tensor(np.concatenate(d), device=dev), maxiter=60, tol=0.0,
                                    precision="f64")
    lay = map_layout(obs)
    for m, (off, npix) in lay.items():
        members = [i for i, o in enumerate(obs) if o.map_id == m]
        sub = [synth.Observation(obs[i].nside, obs[i].q_bore, obs[i].q_det, map_id=0) for i in members]
        Pm = fx.Pointing.from_observations(sub, mode="cache_f64", device=dev)
        Nm = fx.Noise.banded(Pm, np.tile(synth.inverse_noise_taps(), (sum(o.ndet for o in sub), 1)))
        xm, vm, _ = fx.mapmaker_cg(Pm, Nm, torch.as_tensor(np.concatenate([d[i] for i in members]), device=dev),
                                   maxiter=60, tol=0.0, precision="f64")
        assert torch.equal(valid[off:off + npix], vm)
        assert rel(x[off:off + npix].cpu().numpy(), xm.cpu().numpy()) < 1e-12, m


def test_shared_map_needs_equal_nside(fx, dev):
    obs = obs_list([(8, 2, 100), (16, 2, 100)], [1, 1])
    with pytest.raises(fx.FuraxError) as e:
        fx.Pointing.from_observations(obs, mode="cache_f32", device=dev)
    assert e.value.code == -1
