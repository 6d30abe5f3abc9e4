"""GPU operators vs the FP64 oracle: P, P^T (three accumulations), hits, N^-1, block-Jacobi,
the fused normal-equations operator and the right-hand side."""
import numpy as np
import pytest
import torch

import synth
from parity import rel

pytestmark = pytest.mark.gpu




@pytest.fixture(scope="module")
def prob(fx, dev, orc):
    """nside 64, 16 hex detectors, 20000 samples (several tiles + a ragged tail)."""
    o = synth.Observation(64, synth.satellite_scan(20000, t0=100.0), synth.hex_focal_plane(16))
    opix, oc, os_, _ = orc.pointing(o.nside, o.q_bore, o.q_det)
    taps = np.tile(synth.inverse_noise_taps(), (16, 1))
    taps[3] *= 2.0
    sigma2 = np.linspace(80.0, 120.0, 16)
    return o, opix, oc, os_, taps, sigma2


@pytest.mark.parametrize("mode", ["cache_f64", "cache_f32", "on_the_fly"])
def test_P_matches_oracle(fx, dev, orc, prob, mode):
    o, opix, oc, os_, _, _ = prob
    P = fx.Pointing.from_observations([o], mode=mode, device=dev)
    m = synth.gaussian_sky(o.nside, synth.rng(7, 0))
    ref = orc.P(opix, oc, os_, m).ravel()
    got64 = P.apply(torch.as_tensor(m, device=dev), dtype=torch.float64).cpu().numpy()
    if mode == "cache_f32":
        assert rel(got64, ref) < 1e-7
    else:
        assert rel(got64, ref) < 1e-15
    got32 = P.apply(torch.as_tensor(m, device=dev).float()).cpu().numpy()
    assert rel(got32, ref) < 1e-6


@pytest.mark.parametrize("acc,tol", [("f64", 1e-13), ("f32_kahan", 1e-7), ("f32", 1e-5)])
def test_PT_matches_oracle(fx, dev, orc, prob, acc, tol):
    """FP32 modes round each FP64 contribution to FP32 before accumulating (input rounding
    ~6e-8 per term); FP64 accumulates FP64 contributions."""
    o, opix, oc, os_, _, _ = prob
    P = fx.Pointing.from_observations([o], mode="cache_f64", device=dev)
    d = synth.white_noise(16, 20000, synth.rng(7, 1)) + 50.0
    ref, rhits = orc.PT(o.npix, opix, oc, os_, d)
    got, hits = P.transpose(torch.as_tensor(d.ravel(), device=dev), acc=acc, hits=True)
    assert np.array_equal(hits.cpu().numpy(), rhits)
    assert rel(got.cpu().numpy(), ref) < tol
    # accumulate=True adds
    got2 = P.transpose(torch.as_tensor(d.ravel(), device=dev), out=got.clone(), acc=acc, accumulate=True)
    assert rel(got2.cpu().numpy(), 2 * ref) < tol


def test_kahan_accumulation_is_compensated(fx, dev, orc):
    """Nside 1 (12 pixels) and ~1e5 samples per pixel with FP32-exact contributions: the atomic
    two-sum accumulation matches the exact sum to ~1e-10 (the compensation word's own
    rounding), plain FP32 is off by ~sqrt(n) u ~ 1e-5."""
    nd, ns = 8, 200000
    o = synth.Observation(1, synth.satellite_scan(ns), synth.hex_focal_plane(nd))
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    g = np.random.default_rng(5)
    y = (g.integers(-2 ** 20, 2 ** 20, nd * ns) * 2.0 ** -10 + 1000.0).astype(np.float32)
    yt = torch.as_tensor(y, device=dev)
    # I: exact per-pixel sums of the FP32 samples over the oracle's pixels (the cache holds the
    # same pixels, checked bit for bit elsewhere)
    opix, _, _, _ = orc.pointing(1, o.q_bore, o.q_det)
    pn = opix.ravel()
    ok = pn >= 0
    exact_i = np.bincount(pn[ok], y[ok].astype(np.float64), 12)
    k = P.transpose(yt, acc="f32_kahan").cpu().numpy()
    f = P.transpose(yt, acc="f32").cpu().numpy()
    ek = np.abs(k[:, 0] - exact_i).max() / np.abs(exact_i).max()
    ef = np.abs(f[:, 0] - exact_i).max() / np.abs(exact_i).max()
    assert ek < 2e-9
    assert ef > 10 * ek
    # Q, U: the compensated FP32 sums agree with the FP64 accumulation of the same samples to the
    # rounding of the individual contributions (~u / sqrt(n) of the sum)
    d64 = P.transpose(yt, acc="f64").cpu().numpy()
    assert np.abs(k[:, 1:] - d64[:, 1:]).max() / np.abs(d64).max() < 2e-9
    assert np.abs(f[:, 1:] - d64[:, 1:]).max() > 10 * np.abs(k[:, 1:] - d64[:, 1:]).max()


def test_PT_run_twice_same_hits(fx, dev, prob):
    o, *_ = prob
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    ones = torch.ones(P.nsamp_total, dtype=torch.float32, device=dev)
    _, h1 = P.transpose(ones, acc="f32", hits=True)
    _, h2 = P.transpose(ones, acc="f32", hits=True)
    assert torch.equal(h1, h2)


def test_adjoint_identity_gpu(fx, dev, prob):
    o, *_ = prob
    P = fx.Pointing.from_observations([o], mode="cache_f64", device=dev)
    g = torch.Generator(device=dev).manual_seed(3)
    m = torch.randn(P.npix_total, 3, dtype=torch.float64, device=dev, generator=g)
    d = torch.randn(P.nsamp_total, dtype=torch.float64, device=dev, generator=g)
    lhs = torch.dot(P.apply(m), d).item()
    rhs = torch.dot(m.ravel(), P.transpose(d, acc="f64").ravel()).item()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("ns", [1, 62, 63, 64, 127, 4095, 4096, 4097, 9000])
@pytest.mark.parametrize("kind", ["banded", "white"])
def test_noise_inv_matches_oracle(fx, dev, orc, ns, kind):
    nd = 3
    o = synth.Observation(8, synth.satellite_scan(ns), synth.hex_focal_plane(nd))
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    taps = np.tile(synth.inverse_noise_taps(), (nd, 1)) * np.array([[1.0], [0.5], [2.0]])
    sig2 = np.array([100.0, 50.0, 400.0])
    N = fx.Noise.banded(P, taps) if kind == "banded" else fx.Noise.white(P, sig2)
    x = synth.white_noise(nd, ns, synth.rng(8, ns))
    ref = orc.ninv_band(taps, x) if kind == "banded" else orc.ninv_white(sig2, x)
    got64 = N.inv_apply(torch.as_tensor(x.ravel(), device=dev)).cpu().numpy().reshape(nd, ns)
    assert rel(got64, ref) < 1e-14
    got32 = N.inv_apply(torch.as_tensor(x.ravel(), device=dev).float()).cpu().numpy().reshape(nd, ns)
    x32 = x.astype(np.float32).astype(np.float64)
    t32 = taps.astype(np.float32).astype(np.float64)
    ref32 = orc.ninv_band(t32, x32) if kind == "banded" else orc.ninv_white(sig2, x32)
    assert rel(got32, ref32) < 2e-6


@pytest.mark.parametrize("mode", ["cache_f64", "on_the_fly"])
def test_blockdiag_matches_oracle(fx, dev, orc, prob, mode):
    o, opix, oc, os_, taps, _ = prob
    P = fx.Pointing.from_observations([o], mode=mode, device=dev)
    N = fx.Noise.banded(P, taps)
    bj = fx.blockdiag_precond(P, N, 1e-3)
    ref = orc.bj(o.npix, opix, oc, os_, orc.Noise(taps=taps), 1e-3)
    assert np.array_equal(bj["hits"].cpu().numpy(), ref["hits"])
    assert np.array_equal(bj["valid"].cpu().numpy(), ref["valid"])
    assert rel(bj["inv"].cpu().numpy(), ref["inv"]) < 1e-10
    v = ref["valid"]
    assert np.max(np.abs(bj["rcond"].cpu().numpy()[v] - ref["rcond"][v]) / ref["rcond"][v]) < 1e-9


def test_blockdiag_copointed_closed_form(fx, dev):
    obs, _, _, sigma2 = synth.config1(nsamp=65536)
    P = fx.Pointing.from_observations([obs], mode="cache_f32", device=dev)
    bj = fx.blockdiag_precond(P, fx.Noise.white(P, sigma2), 1e-3)
    h = bj["hits"].cpu().numpy()
    v = bj["valid"].cpu().numpy()
    assert np.array_equal(v, h >= 4)
    assert np.allclose(bj["rcond"].cpu().numpy()[v], 0.5, rtol=1e-5)


@pytest.mark.parametrize("noise", ["banded", "white"])
def test_ptnp_apply_matches_oracle(fx, dev, orc, prob, noise):
    o, opix, oc, os_, taps, sigma2 = prob
    P = fx.Pointing.from_observations([o], mode="cache_f64", device=dev)
    N = fx.Noise.banded(P, taps) if noise == "banded" else fx.Noise.white(P, sigma2)
    on = orc.Noise(taps=taps) if noise == "banded" else orc.Noise(sigma2=sigma2)
    bj = orc.bj(o.npix, opix, oc, os_, on)
    valid = bj["valid"]
    x = synth.gaussian_sky(o.nside, synth.rng(7, 2))
    ref = orc.apply_ata(o.npix, opix, oc, os_, on, valid, x)
    vt = torch.as_tensor(valid.astype(np.uint8), device=dev)
    xt = torch.as_tensor(x, device=dev)
    got = fx.ptnp_apply(P, N, xt, vt, precision="f64").cpu().numpy()
    assert rel(got, ref) < 1e-12
    P32 = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    N32 = fx.Noise.banded(P32, taps) if noise == "banded" else fx.Noise.white(P32, sigma2)
    for acc, tol in (("f64", 2e-6), ("f32_kahan", 2e-6), ("f32", 1e-5)):
        got = fx.ptnp_apply(P32, N32, xt, vt, precision="f32", acc=acc).cpu().numpy()
        assert rel(got, ref) < tol, acc
    nomask = orc.apply_ata(o.npix, opix, oc, os_, on, None, x)
    assert rel(fx.ptnp_apply(P, N, xt, None, precision="f64").cpu().numpy(), nomask) < 1e-12


def test_rhs_matches_oracle(fx, dev, orc, prob):
    o, opix, oc, os_, taps, _ = prob
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    N = fx.Noise.banded(P, taps)
    d = synth.one_over_f_noise(16, 20000, synth.rng(7, 3)).astype(np.float32)
    bj = orc.bj(o.npix, opix, oc, os_, orc.Noise(taps=taps))
    # the FP32 cache holds weights within a few 1e-7 of the FP64 ones (the right-hand side itself is
    # FP64-accurate), so Q and U follow to that level and I exactly
    ref = orc.rhs(o.npix, opix, oc, os_, orc.Noise(taps=taps), bj["valid"], d.astype(np.float64))
    got = fx.rhs(P, N, torch.as_tensor(d.ravel(), device=dev),
                 torch.as_tensor(bj["valid"].astype(np.uint8), device=dev)).cpu().numpy()
    assert rel(got[:, 0], ref[:, 0]) < 1e-12
    assert rel(got, ref) < 2e-6


@pytest.mark.parametrize("noise", ["banded", "white"])
@pytest.mark.parametrize("mode", ["cache_mixed", "cache_f64", "on_the_fly"])
def test_double_fp32_operator_is_fp64_accurate(fx, dev, orc, prob, noise, mode):
    """The double-FP32 band product (FP32 pipes) matches the FP64 oracle to FP64-like accuracy
    when the weights are FP64-accurate (mixed hi+lo cache, FP64 cache, on the fly)."""
    o, opix, oc, os_, taps, sigma2 = prob
    P = fx.Pointing.from_observations([o], mode=mode, device=dev)
    N = fx.Noise.banded(P, taps) if noise == "banded" else fx.Noise.white(P, sigma2)
    on = orc.Noise(taps=taps) if noise == "banded" else orc.Noise(sigma2=sigma2)
    valid = orc.bj(o.npix, opix, oc, os_, on)["valid"]
    x = synth.gaussian_sky(o.nside, synth.rng(7, 4))
    ref = orc.apply_ata(o.npix, opix, oc, os_, on, valid, x)
    got = fx.ptnp_apply(P, N, torch.as_tensor(x, device=dev), torch.as_tensor(valid.astype(np.uint8), device=dev),
                        precision="f32x2").cpu().numpy()
    assert rel(got, ref) < 1e-12


def test_mixed_cache_holds_fp64_weights(fx, dev, orc, prob):
    o, opix, oc, os_, *_ = prob
    P = fx.Pointing.from_observations([o], mode="cache_mixed", device=dev)
    pix, c, s = P.expand(torch.float64)
    assert np.array_equal(pix.cpu().numpy().reshape(opix.shape), opix)
    # the FP32 operator of this mode reads the rounded weights, the FP64-accurate ones hi + lo
    m = synth.gaussian_sky(o.nside, synth.rng(7, 5))
    ref = orc.P(opix, oc, os_, m).ravel()
    assert rel(P.apply(torch.as_tensor(m, device=dev), dtype=torch.float64).cpu().numpy(), ref) < 1e-14
    assert rel(P.apply(torch.as_tensor(m, device=dev).float()).cpu().numpy(), ref) < 1e-6


@pytest.fixture(scope="module")
def repeats(orc):
    """nside 256, 4 detectors x 160,000 samples: longer than one precession period, so some
    pixels are crossed only at one angle (singular preconditioner blocks)."""
    o = synth.Observation(256, synth.satellite_scan(160000), synth.hex_focal_plane(4))
    opix, oc, os_, _ = orc.pointing(o.nside, o.q_bore, o.q_det)
    taps = np.tile(synth.inverse_noise_taps(), (4, 1))
    return o, opix, oc, os_, taps


@pytest.mark.parametrize("mode", ["cache_f64", "cache_f32"])
def test_blockdiag_singular_blocks_match_oracle(fx, dev, orc, repeats, mode):
    o, opix, oc, os_, taps = repeats
    P = fx.Pointing.from_observations([o], mode=mode, device=dev)
    bj = fx.blockdiag_precond(P, fx.Noise.banded(P, taps), 1e-2)
    if mode == "cache_f64":
        ref = orc.bj(o.npix, opix, oc, os_, orc.Noise(taps=taps), 1e-2)
        assert np.array_equal(bj["valid"].cpu().numpy(), ref["valid"])
        v = ref["valid"]
        assert rel(bj["inv"].cpu().numpy()[v], ref["inv"][v]) < 1e-10
    v = bj["valid"].cpu().numpy()
    idx = np.array([[0, 1, 2], [1, 3, 4], [2, 4, 5]])
    assert np.all(np.linalg.eigvalsh(bj["inv"].cpu().numpy()[v][:, idx])[:, 0] > 0)


@pytest.mark.parametrize("hwp", [False, True])
def test_on_the_fly_fp32_operator_equals_cached(fx, dev, prob, hwp):
    """The on-the-fly FP32 operator evaluates the pointing with the certified FP32 method of the
    FP32 cache fill (the exact FP64 recipe where the margins cannot certify): pixels and weights,
    hence the operator, equal the cached FP32 operator's up to the order of the FP64 additions;
    with per-detector angle offsets and an ideal half-wave plate too."""
    o, *_ , taps, _ = prob
    w = torch.as_tensor(synth.hwp_angle(o.nsamp), device=dev) if hwp else None
    delta = torch.as_tensor(np.radians(np.linspace(-1.0, 1.0, o.ndet)), device=dev)
    qb = torch.as_tensor(o.q_bore, device=dev)
    qd = torch.as_tensor(o.q_det, device=dev)
    x = torch.as_tensor(synth.gaussian_sky(o.nside, synth.rng(7, 8)), device=dev)
    out = {}
    for mode in ("on_the_fly", "cache_f32"):
        P = fx.Pointing(qb, qd, [o.ndet], [o.nsamp], [o.nside], mode=mode, psi_offset=delta, hwp_angle=w)
        N = fx.Noise.banded(P, taps)
        out[mode] = fx.ptnp_apply(P, N, x, None, "f32", "f64").cpu().numpy()
        P.close()
    assert rel(out["on_the_fly"], out["cache_f32"]) < 1e-12
