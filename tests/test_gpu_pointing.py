"""GPU pointing vs the FP64 oracle: pixels bit-exact, weights to rounding, every storage mode."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _cases():
    # (name, nside, ndet, nsamp, focal plane, psi offsets)
    return [
        ("c1", 16, 4, 65536, "copointed", False),
        ("c2_reduced", 512, 16, 12289, "hex", False),
        ("c3_1024", 1024, 8, 8192, "hex", False),
        ("c5_offsets", 256, 8, 9000, "hex", True),
        ("tiny_ragged", 1, 3, 4097, "hex", False),
    ]


def _obs(nside, ndet, nsamp, fp, offsets, t0=0.0):
    qd = synth.copointed_detectors([0, 45, 90, 135][:ndet]) if fp == "copointed" else synth.hex_focal_plane(ndet)
    o = synth.Observation(nside, synth.satellite_scan(nsamp, t0=t0), qd)
    if offsets:
        o.psi_offset = np.radians(synth.rng(5, 2).normal(0, 1.0, ndet))
    return o


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_expand_matches_oracle(fx, dev, orc, case):
    name, nside, ndet, nsamp, fp, offsets = case
    o = _obs(nside, ndet, nsamp, fp, offsets)
    opix, oc, os_, bad = orc.pointing(nside, o.q_bore, o.q_det, o.psi_offset)
    for mode in ("on_the_fly", "cache_f64", "cache_f32"):
        P = fx.Pointing.from_observations([o], mode=mode, device=dev)
        pix, c, s = P.expand(torch.float64)
        pix = pix.cpu().numpy().reshape(ndet, nsamp)
        assert np.array_equal(pix, opix), f"{mode}: {(pix != opix).sum()} pixel mismatches"
        c = c.cpu().numpy().reshape(ndet, nsamp)
        s = s.cpu().numpy().reshape(ndet, nsamp)
        # identical FP64 recipe: identical bits without offsets; offsets use each side's cos/sin
        tol = 1e-14 if offsets else 0.0
        assert np.max(np.abs(c - oc)) <= tol and np.max(np.abs(s - os_)) <= tol, mode
        pix32, c32, s32 = P.expand(torch.float32)
        assert np.array_equal(pix32.cpu().numpy().reshape(ndet, nsamp), opix)
        if not offsets:
            assert np.array_equal(c32.cpu().numpy().reshape(ndet, nsamp), oc.astype(np.float32))
            assert np.array_equal(s32.cpu().numpy().reshape(ndet, nsamp), os_.astype(np.float32))
        P.close()


def _rho2(orc, qb, qd):
    ns, nd = qb.shape[0], qd.shape[0]
    d, _ = orc.quat_axes(orc.quat_mul(np.tile(qb, (nd, 1)), np.repeat(qd, ns, axis=0)))
    return (d[:, 0] ** 2 + d[:, 1] ** 2).reshape(nd, ns)


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_fp32_cache_matches_oracle(fx, dev, orc, case):
    """The FP32 cache is filled on the FP32 pipes with certified floors and an exact FP64
    fallback: pixels identical to the recipe's, weights within a few 1e-7 (relative error
    ~5 u / rho, with samples closer than rho = 0.05 to a pole recomputed exactly)."""
    name, nside, ndet, nsamp, fp, offsets = case
    o = _obs(nside, ndet, nsamp, fp, False)
    opix, oc, os_, bad = orc.pointing(nside, o.q_bore, o.q_det)
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    pix, c, s = P.cache()
    assert np.array_equal(pix.cpu().numpy().reshape(opix.shape), opix)
    c = c.cpu().numpy().reshape(oc.shape).astype(np.float64)
    s = s.cpu().numpy().reshape(oc.shape).astype(np.float64)
    rho = np.sqrt(np.maximum(_rho2(orc, o.q_bore, o.q_det), 1e-300))
    tol = np.minimum(64 * 2.0 ** -24 / rho, 1e-4) + 2 * 2.0 ** -24
    assert np.all(np.abs(c - oc) <= tol) and np.all(np.abs(s - os_) <= tol)
    P.close()


def test_batched_ragged_expand(fx, dev, orc):
    obs = [_obs(4, 3, 5000, "hex", False), _obs(64, 7, 4096, "hex", False, t0=500.0),
           _obs(16, 1, 1, "hex", False, t0=900.0), _obs(256, 12, 9001, "hex", True, t0=1000.0)]
    P = fx.Pointing.from_observations(obs, mode="cache_f32", device=dev)
    pix, c, s = P.expand(torch.float64)
    pix, c, s = pix.cpu().numpy(), c.cpu().numpy(), s.cpu().numpy()
    off = 0
    for o in obs:
        opix, oc, os_, _ = orc.pointing(o.nside, o.q_bore, o.q_det, o.psi_offset)
        n = opix.size
        assert np.array_equal(pix[off:off + n], opix.ravel())
        assert np.max(np.abs(c[off:off + n] - oc.ravel())) <= 1e-14
        off += n
    assert off == P.nsamp_total


def test_nonfinite_quaternions_are_invalid_samples(fx, dev, orc):
    o = _obs(32, 3, 5000, "hex", False)
    o.q_bore[17, 1] = np.nan
    o.q_bore[4095, 3] = np.inf
    o.q_bore[4096, 0] = -np.inf
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    assert P.n_invalid == 9
    pix, _, _ = P.expand()
    opix, _, _, bad = orc.pointing(32, o.q_bore, o.q_det)
    assert bad == 9
    assert np.array_equal(pix.cpu().numpy().reshape(opix.shape), opix)
    # invalid samples read 0 and add nothing
    m = torch.ones(P.npix_total, 3, dtype=torch.float64, device=dev)
    tod = P.apply(m).cpu().numpy().reshape(opix.shape)
    assert np.all(tod[opix < 0] == 0) and np.all(tod[opix >= 0] != 0)
    _, hits = P.transpose(torch.ones(P.nsamp_total, dtype=torch.float64, device=dev), hits=True)
    assert int(hits.sum()) == P.nsamp_total - 9


def test_full_c2_pointing_sampled(fx, dev, orc):
    """Full 256 x 2^20 focal plane at nside 512, cached FP32: sampled samples against the oracle."""
    ns, nd = 1 << 20, 256
    o = synth.Observation(512, synth.satellite_scan(ns), synth.hex_focal_plane(nd))
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    assert P.n_invalid == 0
    pix, c, s = P.expand(torch.float64)
    g = np.random.default_rng(0)
    dets = g.integers(0, nd, 64)
    for det in dets:
        ts = np.sort(g.choice(ns, 256, replace=False))
        opix, oc, os_, _ = orc.pointing(512, o.q_bore[ts], o.q_det[det:det + 1])
        idx = torch.as_tensor(det * ns + ts, device=dev)
        assert np.array_equal(pix[idx].cpu().numpy(), opix[0])
        assert np.array_equal(c[idx].cpu().numpy(), oc[0])
        assert np.array_equal(s[idx].cpu().numpy(), os_[0])
    # the FP32 cache (certified FP32 floors + exact fallback) holds the recipe's pixel for
    # every one of the 268 M samples
    cpix, _, _ = P.cache()
    assert torch.equal(cpix, pix)
    # hits over the full run: every sample lands on a pixel
    _, hits = P.transpose(torch.ones(P.nsamp_total, dtype=torch.float32, device=dev), acc="f32", hits=True)
    assert int(hits.sum()) == nd * ns


def test_non_unit_quaternions_match_oracle(fx, dev, orc):
    """Scaled quaternions (norms 0.5 .. 3) follow the same recipe on both sides, including the
    rule that a line of sight off the sphere has no pixel."""
    o = _obs(128, 4, 3000, "hex", False)
    scale = np.linspace(0.5, 3.0, 3000)[:, None]
    o.q_bore = np.ascontiguousarray(o.q_bore * scale)
    opix, oc, os_, bad = orc.pointing(128, o.q_bore, o.q_det)
    P = fx.Pointing.from_observations([o], mode="cache_f64", device=dev)
    assert P.n_invalid == bad
    pix, c, s = P.expand()
    assert np.array_equal(pix.cpu().numpy().reshape(opix.shape), opix)
    assert np.array_equal(c.cpu().numpy().reshape(oc.shape), oc)
