"""The pixel-sorted schedule of the cached FP32 normal operator against the oracle.

The sorted kernel groups the detectors that follow one track on the sky into tiles, sorts each
tile's samples by pixel once per refresh, gathers each pixel once per run and accumulates a run
with one (compensated) reduction. It changes the order of the floating-point additions only, so it
is held to the same per-element bound as the time-ordered kernel:
|got - ref| <= (n_band + n_acc) u (|P^T| |N^-1| |P| |x|), u = 2^-24, n_band = 129 (banded) or 2
(white), n_acc = 4 for compensated FP32 and FP64 accumulation and the pixel's hit count + 1 for
plain FP32 (run sums add the same terms in another order). The oracle runs on what the kernel
reads: the GPU's FP32 cache upcast, FP32 taps, powers-of-two inverse variances, the FP32 map."""
import numpy as np
import pytest
import torch

import synth
from parity import elem, rel

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
SHAPES = [(24, 66536, 128), (17, 40003, 64), (23, 70001, 128)]   # > 4 tiles per CTA either way
SCHEDULES = [dict(), dict(tile_len=64, max_rows=4, group_tol=0.5), dict(tile_len=1024, max_rows=3, group_tol=4.0),
             dict(l2_evict_first=1)]


def _pts(P, obs):
    pix, c, s = P.cache()
    pix, c, s = pix.cpu().numpy(), c.cpu().numpy().astype(np.float64), s.cpu().numpy().astype(np.float64)
    out, off = [], 0
    for o in obs:
        n = o.ndet * o.nsamp
        sh = (o.ndet, o.nsamp)
        out.append((pix[off:off + n].reshape(sh), c[off:off + n].reshape(sh), s[off:off + n].reshape(sh)))
        off += n
    return out


def _check(orc, obs, pts, got, taps, sigma2, kind, acc, x, valid, label):
    off, d0 = 0, 0
    for o, (pix, c, s), xi in zip(obs, pts, x):
        vi = None if valid is None else valid[off:off + o.npix]
        if kind == "banded":
            t = taps[d0:d0 + o.ndet]
            on, oa = orc.Noise(taps=t), orc.Noise(taps=np.abs(t))
        else:
            on = oa = orc.Noise(sigma2=sigma2[d0:d0 + o.ndet])
        ref = orc.apply_ata(o.npix, pix, c, s, on, vi, xi)
        scale = orc.apply_ata(o.npix, pix, np.abs(c), np.abs(s), oa, vi, np.abs(xi))
        hits = np.bincount(pix[pix >= 0], minlength=o.npix)
        n_acc = 4 if acc != "f32" else int(hits.max()) + 1
        tol = ((129 if kind == "banded" else 2) + n_acc) * U32
        gi = got[off:off + o.npix]
        assert elem(gi, ref, scale, f"{label}/{o.ndet}x{o.nsamp}") <= tol, (label, o.ndet, o.nsamp)
        if vi is not None:
            assert np.all(gi[~vi] == 0.0)
        off += o.npix
        d0 += o.ndet


@pytest.fixture(scope="module")
def batch(fx, dev):
    obs = [synth.Observation(nside, synth.satellite_scan(ns, t0=211.0 * i), synth.hex_focal_plane(nd))
           for i, (nd, ns, nside) in enumerate(SHAPES)]
    nd = sum(o.ndet for o in obs)
    taps = (np.tile(synth.inverse_noise_taps(), (nd, 1)) * (1.0 + 0.01 * np.arange(nd))[:, None]).astype(np.float32)
    sigma2 = 2.0 ** (4 + np.arange(nd) % 5)
    x = [synth.gaussian_sky(o.nside, synth.rng(82, i)).astype(np.float32).astype(np.float64) for i, o in enumerate(obs)]
    valid = np.concatenate([np.random.default_rng(83 + i).random(o.npix) > 0.05 for i, o in enumerate(obs)])
    return obs, taps.astype(np.float64), sigma2, x, valid


@pytest.mark.parametrize("sched", range(len(SCHEDULES)))
@pytest.mark.parametrize("kind", ["banded", "white"])
@pytest.mark.parametrize("acc", ["f32_kahan", "f64", "f32"])
def test_sorted_operator_matches_oracle(fx, dev, orc, batch, sched, kind, acc):
    obs, taps, sigma2, x, valid = batch
    P = fx.Pointing.from_observations(obs, mode="cache_f32", device=dev)
    P.set_schedule("pixel_sorted", **SCHEDULES[sched])
    assert P.schedule()["kernel"] == "pixel_sorted"
    N = fx.Noise.banded(P, taps) if kind == "banded" else fx.Noise.white(P, sigma2)
    got = fx.ptnp_apply(P, N, torch.as_tensor(np.concatenate(x), device=dev),
                        torch.as_tensor(valid.astype(np.uint8), device=dev), precision="f32", acc=acc).cpu().numpy()
    _check(orc, obs, _pts(P, obs), got, taps, sigma2, kind, acc, x, valid, f"sorted{sched}/{kind}/{acc}")
    P.close()


@pytest.mark.parametrize("kind", ["banded", "white"])
@pytest.mark.parametrize("acc", ["f32_kahan", "f32"])
@pytest.mark.parametrize("kc", [8, 16])
def test_time_ordered_schedules_match_oracle(fx, dev, orc, batch, kind, acc, kc):
    """The L2 evict-first policy on the pointing stream changes only where data are cached; 16
    consumer warps (8 outputs and twice the reductions in flight per thread block) only the split
    of the work."""
    obs, taps, sigma2, x, valid = batch
    P = fx.Pointing.from_observations(obs, mode="cache_f32", device=dev)
    P.set_schedule("time_ordered", l2_evict_first=1, consumer_warps=kc)
    assert P.schedule()["l2_evict_first"] == 1 and P.schedule()["consumer_warps"] == kc
    N = fx.Noise.banded(P, taps) if kind == "banded" else fx.Noise.white(P, sigma2)
    got = fx.ptnp_apply(P, N, torch.as_tensor(np.concatenate(x), device=dev),
                        torch.as_tensor(valid.astype(np.uint8), device=dev), precision="f32", acc=acc).cpu().numpy()
    _check(orc, obs, _pts(P, obs), got, taps, sigma2, kind, acc, x, valid, f"time-ordered l2 kc{kc}/{kind}/{acc}")
    P.close()


def test_sorted_equals_time_ordered_to_rounding(fx, dev, batch):
    """Same operator, other addition order: the compensated results agree to a few FP32 units of the
    band output, far below the operator's own bound."""
    obs, taps, _, x, _ = batch
    P = fx.Pointing.from_observations(obs, mode="cache_f32", device=dev)
    N = fx.Noise.banded(P, taps)
    xt = torch.as_tensor(np.concatenate(x), device=dev)
    a = fx.ptnp_apply(P, N, xt, None, precision="f32", acc="f32_kahan")
    P.set_schedule("pixel_sorted")
    b = fx.ptnp_apply(P, N, xt, None, precision="f32", acc="f32_kahan")
    P.set_schedule("time_ordered")
    c = fx.ptnp_apply(P, N, xt, None, precision="f32", acc="f32_kahan")
    # compensated sums are order-independent to second order only (atomics land in any order)
    assert rel(c, a, "time-ordered run to run") < 1e-9
    assert rel(b, a, "sorted vs time-ordered") < 1e-6


@pytest.mark.parametrize("acc", ["f32_kahan", "f32"])
def test_sorted_with_offsets_plate_and_tiny_streams(fx, dev, orc, acc):
    """Per-detector angle offsets and a rotating half-wave plate (weights rotated in the kernel and
    folded into the cache), on a ragged batch with streams shorter than the band (clipped halos)."""
    shapes = [(3, 1), (2, 5), (4, 63), (3, 64), (2, 127), (5, 4095), (3, 4097), (7, 9001)]
    g = np.random.default_rng(84)
    obs = [synth.Observation(8, synth.satellite_scan(ns, t0=7.0 * i), synth.hex_focal_plane(nd),
                             psi_offset=np.radians(g.normal(0.0, 1.0, nd)), hwp=synth.hwp_angle(ns, t0=7.0 * i))
           for i, (nd, ns) in enumerate(shapes)]
    nd = sum(o.ndet for o in obs)
    taps = np.tile(synth.inverse_noise_taps(), (nd, 1)).astype(np.float32).astype(np.float64)
    P = fx.Pointing.from_observations(obs, mode="cache_f32", device=dev)
    P.set_schedule("pixel_sorted", tile_len=32, max_rows=16, group_tol=8.0)
    N = fx.Noise.banded(P, taps)
    x = [synth.gaussian_sky(8, synth.rng(85, i)).astype(np.float32).astype(np.float64) for i in range(len(obs))]
    got = fx.ptnp_apply(P, N, torch.as_tensor(np.concatenate(x), device=dev), None, precision="f32",
                        acc=acc).cpu().numpy()
    # the cache holds the plate but not the offsets: the oracle sees the weights the kernel uses
    pts = _pts(P, obs)
    rot = []
    d0 = 0
    for o, (pix, c, s) in zip(obs, pts):
        # offsets rotate (c, s) by -2 delta behind the plate
        cd, sd = np.cos(2 * o.psi_offset)[:, None], np.sin(2 * o.psi_offset)[:, None]
        c32, s32 = c.astype(np.float32), s.astype(np.float32)
        cr = (c32 * cd.astype(np.float32) + s32 * sd.astype(np.float32)).astype(np.float64)
        sr = (s32 * cd.astype(np.float32) - c32 * sd.astype(np.float32)).astype(np.float64)
        rot.append((pix, cr, sr))
        d0 += o.ndet
    _check(orc, obs, rot, got, taps, None, "banded", acc, x, None, f"sorted tiny/{acc}")
    P.close()


def test_sorted_follows_refresh(fx, dev, orc):
    """After the boresight changes and the pointing is refreshed, the permutation follows the new
    cache."""
    o = synth.Observation(32, synth.satellite_scan(30000, t0=0.0), synth.hex_focal_plane(19))
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    P.set_schedule("pixel_sorted")
    taps = np.tile(synth.inverse_noise_taps(), (19, 1)).astype(np.float32).astype(np.float64)
    N = fx.Noise.banded(P, taps)
    x = synth.gaussian_sky(32, synth.rng(86, 0)).astype(np.float32).astype(np.float64)
    xt = torch.as_tensor(x, device=dev)
    o2 = synth.Observation(32, synth.satellite_scan(30000, t0=5000.0), o.q_det)
    P.q_bore.copy_(torch.as_tensor(o2.q_bore, device=dev))
    P.refresh()
    got = fx.ptnp_apply(P, N, xt, None, precision="f32", acc="f32_kahan").cpu().numpy()
    _check(orc, [o2], _pts(P, [o2]), got, taps, None, "banded", "f32_kahan", [x], None, "sorted refresh")
    P.close()


def test_sorted_joint_map_and_solver(fx, dev):
    """Observations sharing one map, and the mixed-precision solver: the pixel-sorted schedule
    reaches the time-ordered schedule's solution (same system; the outer correction is FP64-accurate)."""
    obs = [synth.Observation(64, synth.satellite_scan(ns, t0=31.0 * i), synth.hex_focal_plane(nd), map_id=1)
           for i, (nd, ns) in enumerate([(19, 40000), (12, 35001)])]
    taps = np.tile(synth.inverse_noise_taps(), (31, 1))
    g = synth.rng(87, 0)
    d = np.concatenate([(synth.one_over_f_noise(o.ndet, o.nsamp, g)).ravel() for o in obs])
    dt = torch.as_tensor(d.astype(np.float32), device=dev)
    maps = {}
    for sched in ("time_ordered", "pixel_sorted"):
        P = fx.Pointing.from_observations(obs, mode="cache_mixed", device=dev)
        P.set_schedule(sched)
        N = fx.Noise.banded(P, taps)
        x, v, info = fx.mapmaker_cg(P, N, dt, maxiter=400, tol=1e-9, precision="f32", acc="f32_kahan")
        assert info.converged, sched
        maps[sched] = (x.cpu().numpy(), v.cpu().numpy())
        P.close()
    (a, va), (b, vb) = maps["time_ordered"], maps["pixel_sorted"]
    assert np.array_equal(va, vb)
    assert rel(b[vb], a[va], "sorted solve") < 1e-7


def test_sorted_bounded_waits(fx, dev, orc):
    """The sorted kernel's waits are bounded too: with its loader held the launch returns, the
    handle reports FURAX_ETIMEOUT once, and the next launch is correct."""
    from paper_2603_19600_gb300 import _native as nat
    o = synth.Observation(16, synth.satellite_scan(20000, t0=60.0), synth.hex_focal_plane(7))
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    P.set_schedule("pixel_sorted")
    taps = np.tile(synth.inverse_noise_taps(), (7, 1)).astype(np.float32).astype(np.float64)
    N = fx.Noise.banded(P, taps)
    x = synth.gaussian_sky(16, synth.rng(88, 0)).astype(np.float32).astype(np.float64)
    xt = torch.as_tensor(x, device=dev)
    nat.furax_set_wait_budget(P.handle, 1 << 20)
    nat.furax_debug_hold_loader(P.handle, True)
    fx.ptnp_apply(P, N, xt, None, precision="f32", acc="f32_kahan")
    torch.cuda.synchronize()
    with pytest.raises(nat.FuraxError) as e:
        nat.furax_device_status(P.handle)
    assert e.value.code == -5
    nat.furax_debug_hold_loader(P.handle, False)
    nat.furax_set_wait_budget(P.handle, 0)
    got = fx.ptnp_apply(P, N, xt, None, precision="f32", acc="f32_kahan").cpu().numpy()
    nat.furax_device_status(P.handle)
    _check(orc, [o], _pts(P, [o]), got, taps, None, "banded", "f32_kahan", [x], None, "sorted after hold")
    P.close()


def test_schedule_validation(fx, dev):
    from paper_2603_19600_gb300 import _native as nat
    o = synth.Observation(8, synth.satellite_scan(5000), synth.hex_focal_plane(4))
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    assert P.schedule()["kernel"] == "time_ordered"
    for bad in (dict(tile_len=24), dict(tile_len=8192), dict(max_rows=0), dict(max_rows=17), dict(group_tol=0.0),
                dict(l2_evict_first=2), dict(consumer_warps=12)):
        with pytest.raises(nat.FuraxError):
            P.set_schedule("pixel_sorted", **bad)
    P.set_schedule("pixel_sorted", tile_len=128, max_rows=5, group_tol=1.5)
    s = P.schedule()
    assert (s["kernel"], s["tile_len"], s["max_rows"], s["group_tol"]) == ("pixel_sorted", 128, 5, 1.5)
    P64 = fx.Pointing.from_observations([o], mode="cache_f64", device=dev)
    with pytest.raises(nat.FuraxError, match="FP32 pointing cache"):
        P64.set_schedule("pixel_sorted")
    P.close(); P64.close()


def test_autotuned_schedule_keeps_oracle_parity_and_is_cached(fx, dev, orc, batch, tmp_path):
    """The autotuner times candidate schedules on the handle's own workload (compensated
    accumulation, never changed), leaves the fastest set, and stores it: the tuned operator stays
    within the oracle bound, and a second call with the same key sets the stored schedule."""
    obs, taps, sigma2, x, valid = batch
    P = fx.Pointing.from_observations(obs, mode="cache_f32", device=dev)
    N = fx.Noise.banded(P, taps)
    space = fx._native.furax_autotune_space()
    assert space[0]["kernel"] == 0 and len(space) > 10
    cache = str(tmp_path / "schedules.json")
    r = fx.autotune(P, N, "f32_kahan", reps=2, cache_path=cache, candidates=space[:1] + space[1::6])
    assert not r["cached"] and r["candidates_timed"] >= 2
    assert P.schedule()["kernel"] == r["schedule"]["kernel"]
    got = fx.ptnp_apply(P, N, torch.as_tensor(np.concatenate(x), device=dev),
                        torch.as_tensor(valid.astype(np.uint8), device=dev), precision="f32",
                        acc="f32_kahan").cpu().numpy()
    _check(orc, obs, _pts(P, obs), got, taps, sigma2, "banded", "f32_kahan", x, valid, "autotuned")
    P.set_schedule("time_ordered")
    r2 = fx.autotune(P, N, "f32_kahan", cache_path=cache)
    assert r2["cached"] and r2["schedule"] == r["schedule"]
    s = P.schedule()
    assert (s["kernel"], s["tile_len"], s["max_rows"]) == (r["schedule"]["kernel"], r["schedule"]["tile_len"],
                                                           r["schedule"]["max_rows"])
    P.close()
