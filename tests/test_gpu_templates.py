"""Template deprojection on the GPU (F_T = W - W T (T^T W T)^-1 T^T W; Statement of Need,
TemplateOperator of Table 3) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import synth
from parity import rel
from oracle import templates as ot

pytestmark = pytest.mark.gpu




# ragged batch: streams shorter than the band, one tile, several tiles with a ragged tail
SHAPES = [(2, 40), (3, 200), (2, 4096), (4, 9001)]


@pytest.fixture(scope="module")
def batch(orc):
    obs = [synth.Observation(8, synth.satellite_scan(ns, t0=13.0 * i), synth.hex_focal_plane(nd))
           for i, (nd, ns) in enumerate(SHAPES)]
    taps = [np.tile(synth.inverse_noise_taps(), (o.ndet, 1)) * (1.0 + 0.2 * np.arange(o.ndet))[:, None] for o in obs]
    pts = [orc.pointing(o.nside, o.q_bore, o.q_det)[:3] for o in obs]
    return obs, taps, pts


def split_tod(obs, y):
    out, off = [], 0
    for o in obs:
        out.append(y[off:off + o.ndet * o.nsamp].reshape(o.ndet, o.nsamp))
        off += o.ndet * o.nsamp
    return out


@pytest.mark.parametrize("order", [0, 1, 2, 3])
@pytest.mark.parametrize("kind", ["banded", "white"])
def test_gram_matches_oracle(fx, dev, orc, batch, order, kind):
    obs, taps, _ = batch
    P = fx.Pointing.from_observations(obs, mode="cache_f32", device=dev)
    if kind == "banded":
        N = fx.Noise.banded(P, np.concatenate(taps))
        on = [orc.Noise(taps=t) for t in taps]
    else:
        s2 = [np.linspace(50.0, 150.0, o.ndet) for o in obs]
        N = fx.Noise.white(P, np.concatenate(s2))
        on = [orc.Noise(sigma2=s) for s in s2]
    T = fx.Templates(P, N, order)
    g = T.gram().cpu().numpy()
    off = 0
    for o, n in zip(obs, on):
        ref = ot.gram(n, o.ndet, o.nsamp, order)
        assert rel(g[off:off + o.ndet], ref) < 1e-12, (o.ndet, o.nsamp)
        off += o.ndet


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-11), (torch.float32, 2e-5)])
@pytest.mark.parametrize("order", [0, 3])
def test_deproject_tod_matches_oracle(fx, dev, orc, batch, dtype, tol, order):
    obs, taps, _ = batch
    P = fx.Pointing.from_observations(obs, mode="cache_f32", device=dev)
    N = fx.Noise.banded(P, np.concatenate(taps))
    T = fx.Templates(P, N, order)
    g = np.random.default_rng(1)
    xs = [g.normal(size=(o.ndet, o.nsamp)) + 30.0 * ot.legendre_templates(o.nsamp, min(order, 1))[:, -1] for o in obs]
    x = np.concatenate([a.ravel() for a in xs])
    if dtype == torch.float32:
        x = x.astype(np.float32).astype(np.float64)   # the oracle sees the same FP32 inputs
    y = T.deproject(torch.as_tensor(x, device=dev, dtype=dtype)).double().cpu().numpy()
    for o, t, xi, yi in zip(obs, taps, split_tod(obs, x), split_tod(obs, y)):
        ref = ot.deproject(orc.Noise(taps=t), order, xi)
        assert rel(yi, ref) < tol, (o.ndet, o.nsamp)


def test_templates_are_annihilated_on_gpu(fx, dev, batch):
    """F_T T = 0 (FP64): a TOD made only of templates deprojects to rounding noise."""
    obs, taps, _ = batch
    P = fx.Pointing.from_observations(obs, mode="cache_f64", device=dev)
    N = fx.Noise.banded(P, np.concatenate(taps))
    T = fx.Templates(P, N, 3)
    g = np.random.default_rng(2)
    x = np.concatenate([(g.normal(size=(o.ndet, 4)) * 100 @ ot.legendre_templates(o.nsamp, 3).T).ravel()
                        for o in obs])
    xt = torch.as_tensor(x, device=dev)
    y = T.deproject(xt).cpu().numpy()
    z = torch.empty_like(xt)
    fx._native.furax_noise_inv_apply(N.handle, xt, z)
    assert np.abs(y).max() < 1e-11 * np.abs(z.cpu().numpy()).max()


@pytest.mark.parametrize("mode,prec,acc,tol", [("cache_f64", "f64", "f64", 1e-11), ("on_the_fly", "f64", "f64", 1e-11),
                                               ("cache_mixed", "f32x2", "f64", 1e-11),
                                               ("cache_f32", "f32", "f64", 3e-6), ("cache_f32", "f32", "f32", 1e-5),
                                               ("cache_f32", "f32", "f32_kahan", 3e-6)])
def test_ptfp_apply_matches_oracle(fx, dev, orc, batch, mode, prec, acc, tol):
    obs, taps, pts = batch
    order = 2
    P = fx.Pointing.from_observations(obs, mode=mode, device=dev)
    N = fx.Noise.banded(P, np.concatenate(taps))
    T = fx.Templates(P, N, order)
    g = np.random.default_rng(3)
    x = [synth.gaussian_sky(o.nside, synth.rng(30, i)) for i, o in enumerate(obs)]
    valid = [g.random(o.npix) > 0.1 for o in obs]
    got = fx.ptfp_apply(T, torch.as_tensor(np.concatenate(x), device=dev),
                        torch.as_tensor(np.concatenate(valid), device=dev), precision=prec, acc=acc).cpu().numpy()
    off = 0
    for o, t, (pix, c, s), xi, vi in zip(obs, taps, pts, x, valid):
        ref = ot.ptfp_apply(o.npix, pix, c, s, orc.Noise(taps=t), order, vi, xi)
        assert rel(got[off:off + o.npix], ref) < tol, (o.ndet, o.nsamp)
        off += o.npix


@pytest.mark.parametrize("order", [0, 1, 3])
@pytest.mark.parametrize("kind", ["banded", "white", "long"])
@pytest.mark.parametrize("precision,mode", [("f32", "cache_mixed"), ("f32", "on_the_fly"), ("f64", "cache_f64")])
def test_deprojected_rhs_matches_oracle(fx, dev, orc, batch, order, kind, precision, mode):
    """The deprojected right-hand side S P^T F_T d of FP32 data, seen through the binned map
    M^-1 b. The mixed solver subtracts (W T) b inside its double-FP32 pass over d (a cubic per
    tile in the interior, term by term at the stream ends); the FP64 solver, and any solver with a
    long (overlap-save) band, in a pass of its own. Large drifts along every Legendre degree make
    the correction the dominant term."""
    obs, taps, pts = batch
    P = fx.Pointing.from_observations(obs, mode=mode, device=dev)
    if kind in ("banded", "long"):
        if kind == "long":   # 300 taps: streams of 40 and 200 samples lie wholly within a half-band of an end
            taps = [np.tile(synth.inverse_noise_taps(300), (o.ndet, 1)) * (1.0 + 0.2 * np.arange(o.ndet))[:, None]
                    for o in obs]
        N = fx.Noise.banded(P, np.concatenate(taps))
        on = [orc.Noise(taps=t) for t in taps]
    else:
        s2 = [np.linspace(50.0, 150.0, o.ndet) for o in obs]
        N = fx.Noise.white(P, np.concatenate(s2))
        on = [orc.Noise(sigma2=s) for s in s2]
    T = fx.Templates(P, N, order)
    g = synth.rng(32, order)
    d = [(g.normal(size=(o.ndet, o.nsamp)) + g.normal(size=(o.ndet, 4)) * 300.0 @ ot.legendre_templates(o.nsamp, 3).T)
         .astype(np.float32) for o in obs]
    x, valid, _ = fx.mapmaker_cg(P, N, torch.as_tensor(np.concatenate([di.ravel() for di in d]), device=dev),
                                 binned_only=True, precision=precision, templates=T)
    x, valid = x.cpu().numpy(), valid.cpu().numpy()
    off = 0
    for o, n, (pix, c, s), di in zip(obs, on, pts, d):
        bjd = orc.bj(o.npix, pix, c, s, n)
        v = bjd["valid"]
        ref = orc.binned_map(bjd, ot.rhs(o.npix, pix, c, s, n, order, v, di.astype(np.float64)))
        assert np.array_equal(valid[off:off + o.npix], v)
        assert rel(x[off:off + o.npix][v], ref[v]) < 1e-10, (o.ndet, o.nsamp)
        off += o.npix


@pytest.fixture(scope="module")
def solve_case(orc):
    """nside 8, 12 detectors x 12000 samples, 1/f + white noise, order-2 templates with large
    per-detector drifts added to the data."""
    o = synth.Observation(8, synth.satellite_scan(12000, t0=5.0), synth.hex_focal_plane(12))
    pix, c, s, _ = orc.pointing(o.nside, o.q_bore, o.q_det)
    taps = np.tile(synth.inverse_noise_taps(), (12, 1))
    g = synth.rng(31, 0)
    sky = synth.gaussian_sky(o.nside, g)
    d = orc.P(pix, c, s, sky) + synth.one_over_f_noise(12, 12000, g)
    d = d + g.normal(size=(12, 3)) * 200.0 @ ot.legendre_templates(12000, 2).T
    d = d.astype(np.float32).astype(np.float64)
    on = orc.Noise(taps=taps)
    bjd = orc.bj(o.npix, pix, c, s, on, rcond_min=1e-3)
    b = ot.rhs(o.npix, pix, c, s, on, 2, bjd["valid"], d)
    xo, it, hist = ot.pcg(o.npix, pix, c, s, on, 2, bjd["valid"], bjd["inv"], b, 500, 1e-11)
    assert hist[-1] <= 1e-11
    return o, pix, c, s, taps, d, bjd, xo


def demono(m, v):
    m = m[v].copy()
    m[:, 0] -= m[:, 0].mean()
    return m


@pytest.mark.parametrize("precision,mode,tol", [("f64", "cache_f64", 1e-7), ("f32", "cache_mixed", 1e-6),
                                                ("f32", "cache_f32", 1e-5)])
def test_deprojected_solve_matches_oracle(fx, dev, orc, solve_case, precision, mode, tol):
    """Converged maps (I monopole removed: it is the near-null direction of the offset templates).
    The FP32 cache holds weights within a few 1e-7 of the FP64 ones, hence its looser bound."""
    o, pix, c, s, taps, d, bjd, xo = solve_case
    P = fx.Pointing.from_observations([o], mode=mode, device=dev)
    N = fx.Noise.banded(P, taps)
    T = fx.Templates(P, N, 2)
    dt = torch.as_tensor(d.ravel().astype(np.float32), device=dev)
    x, valid, info = fx.mapmaker_cg(P, N, dt, maxiter=500, tol=1e-10, precision=precision, templates=T)
    assert info.converged and info.true_rel_res <= 1e-10
    v = valid.cpu().numpy()
    assert np.array_equal(v, bjd["valid"])
    assert rel(demono(x.cpu().numpy(), v), demono(xo, v)) < tol


@pytest.mark.parametrize("precision,mode,tol", [("f64", "cache_f64", 1e-8), ("f32", "cache_f32", 1e-5)])
def test_noiseless_data_recovers_map_and_amplitudes(fx, dev, orc, solve_case, precision, mode, tol):
    """d = P m0 + T alpha (m0 zero on unsolved pixels): the solve returns m0 plus a constant I
    offset delta on the solved pixels, and the amplitudes alpha - delta e_0 (the offsets absorb
    what the map's monopole gives up)."""
    o, pix, c, s, taps, _, bjd, _ = solve_case
    v = bjd["valid"]
    m0 = np.where(v[:, None], synth.gaussian_sky(o.nside, synth.rng(32, 0)), 0.0)
    alpha = np.random.default_rng(10).normal(size=(12, 3)) * 300.0
    d = orc.P(pix, c, s, m0) + alpha @ ot.legendre_templates(12000, 2).T
    P = fx.Pointing.from_observations([o], mode=mode, device=dev)
    N = fx.Noise.banded(P, taps)
    T = fx.Templates(P, N, 2)
    amp = torch.empty(12, 3, dtype=torch.float64, device=dev)
    x, valid, info = fx.mapmaker_cg(P, N, torch.as_tensor(d.ravel(), device=dev), maxiter=500, tol=1e-12,
                                    precision=precision, templates=T, amplitudes=amp)
    assert np.array_equal(valid.cpu().numpy(), v)
    xg = x.cpu().numpy()
    delta = np.mean(xg[v, 0] - m0[v, 0])
    scale = np.abs(m0).max()
    assert np.abs(xg[v, 0] - m0[v, 0] - delta).max() < tol * scale
    assert np.abs(xg[v, 1:] - m0[v, 1:]).max() < tol * scale
    a = amp.cpu().numpy()
    assert np.abs(a[:, 1:] - alpha[:, 1:]).max() < tol * scale
    assert np.abs(a[:, 0] - (alpha[:, 0] - delta)).max() < tol * scale


def test_solve_is_invariant_under_template_contamination(fx, dev, solve_case):
    """d -> d + T alpha leaves the deprojected map unchanged (F_T T = 0), GPU only."""
    o, pix, c, s, taps, d, _, _ = solve_case
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    N = fx.Noise.banded(P, taps)
    T = fx.Templates(P, N, 2)
    g = np.random.default_rng(9)
    d2 = d + g.normal(size=(12, 3)) * 500.0 @ ot.legendre_templates(12000, 2).T
    x1, v1, _ = fx.mapmaker_cg(P, N, torch.as_tensor(d.ravel(), device=dev), maxiter=300, tol=1e-11, precision="f64",
                               templates=T)
    x2, v2, _ = fx.mapmaker_cg(P, N, torch.as_tensor(d2.ravel(), device=dev), maxiter=300, tol=1e-11,
                               precision="f64", templates=T)
    v = v1.cpu().numpy()
    assert rel(demono(x2.cpu().numpy(), v), demono(x1.cpu().numpy(), v)) < 1e-7


def test_invalid_template_setups_are_rejected(fx, dev):
    o = synth.Observation(8, synth.satellite_scan(3), synth.hex_focal_plane(2))
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    N = fx.Noise.white(P, np.ones(2))
    with pytest.raises(fx.FuraxError) as e:
        fx.Templates(P, N, 3)
    assert e.value.code == -4
    with pytest.raises(fx.FuraxError) as e:
        fx.Templates(P, N, 4)
    assert e.value.code == -1
    T = fx.Templates(P, N, 2)   # three samples carry three templates
    assert T.gram().shape == (2, 3, 3)


def test_full_size_gram_and_annihilation_sampled(fx, dev, orc):
    """256 detectors x 2^20 samples, banded W, order 1: Gram matrices of sampled detectors against
    the oracle, and F_T T = 0 over the whole TOD."""
    ns, nd = 1 << 20, 256
    o = synth.Observation(512, synth.satellite_scan(ns), synth.hex_focal_plane(nd))
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    taps = np.tile(synth.inverse_noise_taps(), (nd, 1)) * np.linspace(0.5, 2.0, nd)[:, None]
    N = fx.Noise.banded(P, taps)
    T = fx.Templates(P, N, 1)
    g = T.gram().cpu().numpy()
    for det in (0, 77, 255):
        ref = ot.gram(orc.Noise(taps=taps[det:det + 1]), 1, ns, 1)[0]
        # 2^20-term FP64 sums on both sides: the recursive-summation bound n u = 2^20 2^-53
        assert rel(g[det], ref) < 2.0 ** 20 * 2.0 ** -53
    L = torch.as_tensor(ot.legendre_templates(ns, 1), device=dev)
    alpha = torch.randn(nd, 2, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(4))
    x = (alpha @ L.T).reshape(-1).contiguous()
    y = T.deproject(x)
    z = torch.empty_like(x)
    fx._native.furax_noise_inv_apply(N.handle, x, z)
    assert float(y.abs().max()) < 1e-11 * float(z.abs().max())


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_mixed_deprojected_solve_reaches_the_fp64_solve(fx, dev, order):
    """The mixed solve (inner FP32 iterations on the augmented system [map; amplitudes] for
    order <= 2, on the explicit correction for order 3) reaches the FP64 solve of the deprojected
    system; the two observations share one map."""
    obs = [synth.Observation(8, synth.satellite_scan(ns, t0=31.0 * i), synth.hex_focal_plane(nd), map_id=1)
           for i, (nd, ns) in enumerate([(5, 9000), (4, 7000)])]
    taps = np.tile(synth.inverse_noise_taps(), (9, 1))
    g = synth.rng(33, order)
    d = np.concatenate([(synth.one_over_f_noise(o.ndet, o.nsamp, g)
                         + g.normal(size=(o.ndet, 3)) * 100.0 @ ot.legendre_templates(o.nsamp, 2).T).ravel()
                        for o in obs])
    P = fx.Pointing.from_observations(obs, mode="cache_mixed", device=dev)
    N = fx.Noise.banded(P, taps)
    T = fx.Templates(P, N, order)
    dt = torch.as_tensor(d.astype(np.float32), device=dev)
    x64, v64, i64 = fx.mapmaker_cg(P, N, dt, maxiter=500, tol=1e-10, precision="f64", templates=T)
    x32, v32, i32 = fx.mapmaker_cg(P, N, dt, maxiter=500, tol=1e-10, precision="f32", templates=T)
    assert i64.converged and i32.converged and i32.true_rel_res <= 1e-10
    v = v64.cpu().numpy()
    assert np.array_equal(v, v32.cpu().numpy())
    assert rel(demono(x32.cpu().numpy(), v), demono(x64.cpu().numpy(), v)) < 1e-7
