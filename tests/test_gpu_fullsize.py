"""The cached FP32 normal operator in its steady state, element by element against the oracle.

The persistent fused kernel walks the tile list with one CTA per SM and hands tiles between its
roles through two-stage rings; a stage is reused, with the other phase parity, from a CTA's third
tile on. The batch here has more than four tiles per CTA (ragged observations whose tiles straddle
CTAs), so every CTA runs the reuse path that the full-size workload runs, in every accumulation
mode, with white and banded noise, and with the template projection folded into the kernel.

The oracle runs on exactly what the kernel reads: the pixels and FP32 weights of the GPU's cache
(upcast), the FP32-rounded map and FP32 taps, and inverse variances that are powers of two, so the
remaining differences are the kernel's FP32 arithmetic. Bound per element (standard rounding-error
analysis, u = 2^-24): |got - ref| <= (n_band + n_acc) u (|P^T| |N^-1| |P| |x|), with n_band = 2 + 127
(gather FMAs and the 127-term band product; 2 for white noise) and n_acc = 4 for compensated FP32
or FP64 accumulation, the pixel's hit count for plain FP32 accumulation. The scale |P^T||N^-1||P||x|
is the oracle's own operator applied to absolute values.
"""
import numpy as np
import pytest
import torch

import synth
from parity import elem, rel

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
# (ndet, nsamp, nside): tiles = ndet * ceil(nsamp / 4096) = 408 + 170 + 414 = 992 > 4 x 152
SHAPES = [(24, 66536, 128), (17, 40003, 64), (23, 70001, 128)]


@pytest.fixture(scope="module")
def big(fx, dev, orc):
    obs = [synth.Observation(nside, synth.satellite_scan(ns, t0=211.0 * i), synth.hex_focal_plane(nd))
           for i, (nd, ns, nside) in enumerate(SHAPES)]
    P = fx.Pointing.from_observations(obs, mode="cache_f32", device=dev)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    n_tiles = sum(nd * -(-ns // 4096) for nd, ns, _ in SHAPES)
    assert n_tiles >= 4 * n_sm, (n_tiles, n_sm)
    pix, c, s = P.cache()
    pix, c, s = pix.cpu().numpy(), c.cpu().numpy().astype(np.float64), s.cpu().numpy().astype(np.float64)
    pts, off = [], 0
    for o in obs:
        n = o.ndet * o.nsamp
        pts.append((pix[off:off + n].reshape(o.ndet, o.nsamp), c[off:off + n].reshape(o.ndet, o.nsamp),
                    s[off:off + n].reshape(o.ndet, o.nsamp)))
        off += n
    nd = sum(o.ndet for o in obs)
    taps = (np.tile(synth.inverse_noise_taps(), (nd, 1)) * (1.0 + 0.01 * np.arange(nd))[:, None]).astype(np.float32)
    sigma2 = 2.0 ** (4 + np.arange(nd) % 5)   # powers of two: 1/sigma^2 is exact in FP32
    g = np.random.default_rng(77)
    x = [synth.gaussian_sky(o.nside, synth.rng(80, i)).astype(np.float32).astype(np.float64) for i, o in enumerate(obs)]
    valid = [g.random(o.npix) > 0.05 for o in obs]
    return dict(obs=obs, P=P, pts=pts, taps=taps.astype(np.float64), sigma2=sigma2, x=x, valid=valid)


def _split(obs, arr, per):
    out, off = [], 0
    for o in obs:
        n = per(o)
        out.append(arr[off:off + n])
        off += n
    return out


def _noise(orc, big, kind, lo, hi, absolute=False):
    if kind == "banded":
        t = big["taps"][lo:hi]
        return orc.Noise(taps=np.abs(t) if absolute else t)
    return orc.Noise(sigma2=big["sigma2"][lo:hi])


@pytest.mark.parametrize("kind", ["banded", "white"])
@pytest.mark.parametrize("acc", ["f32_kahan", "f64", "f32"])
def test_fused_operator_steady_state_matches_oracle(fx, dev, orc, big, kind, acc):
    obs, P = big["obs"], big["P"]
    N = fx.Noise.banded(P, big["taps"]) if kind == "banded" else fx.Noise.white(P, big["sigma2"])
    xt = torch.as_tensor(np.concatenate(big["x"]), device=dev)
    vt = torch.as_tensor(np.concatenate(big["valid"]).astype(np.uint8), device=dev)
    got = fx.ptnp_apply(P, N, xt, vt, precision="f32", acc=acc).cpu().numpy()
    gots = _split(obs, got, lambda o: o.npix)
    d0 = 0
    n_band = 129 if kind == "banded" else 2
    for o, (pix, c, s), xi, vi, gi in zip(obs, big["pts"], big["x"], big["valid"], gots):
        on = _noise(orc, big, kind, d0, d0 + o.ndet)
        ref = orc.apply_ata(o.npix, pix, c, s, on, vi, xi)
        scale = orc.apply_ata(o.npix, pix, np.abs(c), np.abs(s), _noise(orc, big, kind, d0, d0 + o.ndet, True), vi,
                              np.abs(xi))
        hits = np.bincount(pix[pix >= 0], minlength=o.npix)
        n_acc = 4 if acc != "f32" else int(hits.max()) + 1
        tol = (n_band + n_acc) * U32
        assert elem(gi, ref, scale, f"{kind}/{acc}/{o.ndet}x{o.nsamp}") <= tol, (o.ndet, o.nsamp)
        # masked pixels are exactly zero
        assert np.all(gi[~vi] == 0.0)
        d0 += o.ndet


@pytest.mark.parametrize("acc", ["f32_kahan", "f64"])
def test_fused_operator_steady_state_with_template_projection(fx, dev, orc, big, acc):
    """The template projection T^T N^-1 P x reduced inside the fused kernel (degree <= 2 Legendre
    templates per detector), on the same steady-state batch, against the oracle's explicit F_T."""
    from oracle import templates as ot
    obs, P = big["obs"], big["P"]
    N = fx.Noise.banded(P, big["taps"])
    T = fx.Templates(P, N, 2)
    xt = torch.as_tensor(np.concatenate(big["x"]), device=dev)
    vt = torch.as_tensor(np.concatenate(big["valid"]).astype(np.uint8), device=dev)
    got = fx.ptfp_apply(T, xt, vt, precision="f32", acc=acc).cpu().numpy()
    gots = _split(obs, got, lambda o: o.npix)
    d0 = 0
    for o, (pix, c, s), xi, vi, gi in zip(obs, big["pts"], big["x"], big["valid"], gots):
        ref = ot.ptfp_apply(o.npix, pix, c, s, orc.Noise(taps=big["taps"][d0:d0 + o.ndet]), 2, vi, xi)
        # the projection sums a whole stream (up to 7e4 terms) per detector in FP32 partial sums
        # before FP64: component-scaled bound
        assert rel(gi, ref, f"tpl/{acc}/{o.ndet}x{o.nsamp}") < 5e-6, (o.ndet, o.nsamp)
        d0 += o.ndet
    T.close()


def test_fused_operator_steady_state_is_run_to_run_consistent(fx, dev, big):
    """Compensated accumulation is order-independent to second order: two applications of the same
    input agree far below the FP32 rounding of a single contribution."""
    P = big["P"]
    N = fx.Noise.banded(P, big["taps"])
    xt = torch.as_tensor(np.concatenate(big["x"]), device=dev)
    a = fx.ptnp_apply(P, N, xt, None, precision="f32", acc="f32_kahan")
    b = fx.ptnp_apply(P, N, xt, None, precision="f32", acc="f32_kahan")
    assert rel(a, b, "kahan run-to-run") < 1e-9


def test_augmented_template_solve_steady_state(fx, dev):
    """The augmented inner system of the mixed deprojected solve (amplitudes fetched by the loader
    with each tile, one pseudo-pixel per detector) at more than four tiles per CTA: the mixed solve
    reaches the FP64 solve of the same deprojected system."""
    from oracle import templates as ot
    obs = [synth.Observation(64, synth.satellite_scan(ns, t0=17.0 * i), synth.hex_focal_plane(nd), map_id=1)
           for i, (nd, ns) in enumerate([(40, 50000), (24, 47001)])]
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    assert 40 * 13 + 24 * 12 >= 4 * n_sm
    taps = np.tile(synth.inverse_noise_taps(), (64, 1))
    g = synth.rng(81, 0)
    d = np.concatenate([(synth.one_over_f_noise(o.ndet, o.nsamp, g)
                         + g.normal(size=(o.ndet, 3)) * 100.0 @ ot.legendre_templates(o.nsamp, 2).T).ravel()
                        for o in obs])
    P = fx.Pointing.from_observations(obs, mode="cache_mixed", device=dev)
    N = fx.Noise.banded(P, taps)
    T = fx.Templates(P, N, 2)
    dt = torch.as_tensor(d.astype(np.float32), device=dev)
    x64, v64, i64 = fx.mapmaker_cg(P, N, dt, maxiter=500, tol=1e-10, precision="f64", templates=T)
    x32, v32, i32 = fx.mapmaker_cg(P, N, dt, maxiter=500, tol=1e-10, precision="f32", acc="f32_kahan", templates=T)
    assert i64.converged and i32.converged and i32.true_rel_res <= 1e-10
    v = v64.cpu().numpy()
    assert np.array_equal(v, v32.cpu().numpy())
    a, b = x32.cpu().numpy()[v], x64.cpu().numpy()[v]
    a[:, 0] -= a[:, 0].mean()
    b[:, 0] -= b[:, 0].mean()
    assert rel(a, b, "augmented steady state") < 1e-6
    T.close()
