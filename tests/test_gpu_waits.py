"""Bounded device waits of the pipelined FP32 operator.

Every mbarrier wait between the kernel's roles gives up after a budget of SM cycles: it sets the
handle's error word and its role leaves the loop, so the kernel returns with the context intact.
Here the loader is held back (it issues no copy, so nothing is ever in flight) and the budget is
short: the launch returns within milliseconds, furax_device_status reports FURAX_ETIMEOUT once and
clears the word, the solver reports it at its next synchronisation, and the next normal launch
matches the oracle. No trap, no fault, no wait left without an end."""
import time

import numpy as np
import pytest
import torch

import synth
from parity import elem, rel

pytestmark = pytest.mark.gpu

ETIMEOUT = -5


@pytest.fixture(scope="module")
def case(fx, dev, orc):
    o = synth.Observation(16, synth.satellite_scan(20000, t0=50.0), synth.hex_focal_plane(4))
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    taps = np.tile(synth.inverse_noise_taps(), (4, 1)).astype(np.float32).astype(np.float64)
    N = fx.Noise.banded(P, taps)
    x = synth.gaussian_sky(16, synth.rng(90, 0)).astype(np.float32).astype(np.float64)
    pix, c, s = (a.cpu().numpy() for a in P.cache())
    shp = (o.ndet, o.nsamp)
    pts = (pix.reshape(shp), c.astype(np.float64).reshape(shp), s.astype(np.float64).reshape(shp))
    ref = orc.apply_ata(o.npix, *pts, orc.Noise(taps=taps), None, x)
    scale = orc.apply_ata(o.npix, pts[0], np.abs(pts[1]), np.abs(pts[2]), orc.Noise(taps=np.abs(taps)), None, np.abs(x))
    yield o, P, N, x, ref, scale
    from paper_2603_19600_gb300 import _native as nat
    nat.furax_debug_hold_loader(P.handle, False)
    nat.furax_set_wait_budget(P.handle, 0)


def test_wait_runs_out_and_the_next_call_is_correct(fx, dev, case):
    from paper_2603_19600_gb300 import _native as nat
    o, P, N, x, ref, scale = case
    xt = torch.as_tensor(x, device=dev)
    nat.furax_device_status(P.handle)                      # clean before
    good = fx.ptnp_apply(P, N, xt, None, "f32", "f32_kahan").cpu().numpy()
    nat.furax_device_status(P.handle)                      # a normal launch sets nothing
    assert elem(good, ref, scale, "before hold") <= 140 * 2.0 ** -24

    nat.furax_set_wait_budget(P.handle, 1 << 20)           # ~0.5-1 ms per wait
    nat.furax_debug_hold_loader(P.handle, True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fx.ptnp_apply(P, N, xt, None, "f32", "f32_kahan")
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 2.0                  # the kernel returned by itself
    with pytest.raises(nat.FuraxError) as e:
        nat.furax_device_status(P.handle)
    assert e.value.code == ETIMEOUT
    nat.furax_device_status(P.handle)                      # reported once, then cleared

    # the solver sees it at its next synchronisation point
    d = torch.as_tensor(synth.one_over_f_noise(o.ndet, o.nsamp, synth.rng(90, 1)).ravel().astype(np.float32),
                        device=dev)
    with pytest.raises(nat.FuraxError) as e:
        fx.mapmaker_cg(P, N, d, maxiter=20, tol=1e-8, precision="f32", acc="f32_kahan", check_every=5)
    assert e.value.code == ETIMEOUT
    with pytest.raises(nat.FuraxError):
        nat.furax_device_status(P.handle)                  # the word the solver saw, cleared here

    nat.furax_debug_hold_loader(P.handle, False)
    nat.furax_set_wait_budget(P.handle, 0)
    after = fx.ptnp_apply(P, N, xt, None, "f32", "f32_kahan").cpu().numpy()
    nat.furax_device_status(P.handle)
    assert elem(after, ref, scale, "after hold") <= 140 * 2.0 ** -24
    assert rel(after, good, "after vs before") < 1e-9
    x_, _, info = fx.mapmaker_cg(P, N, d, maxiter=200, tol=1e-8, precision="f32", acc="f32_kahan")
    assert info.converged


def test_wait_budget_is_validated(fx, dev, case):
    from paper_2603_19600_gb300 import _native as nat
    _, P, *_ = case
    with pytest.raises(nat.FuraxError):
        nat.furax_set_wait_budget(P.handle, -1)
