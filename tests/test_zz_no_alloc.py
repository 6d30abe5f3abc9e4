"""The allocation-free normal-equations operator (for callers that cannot allocate device
memory, e.g. inside a pre-sized memory pool) against the regular entry point.

Collected last on purpose: a failure here leaves every other test already run. It must pass both
alone in a fresh process (the first call sets up the static scratch) and after the other tests."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_ptnp_apply_twice(fx, dev):
    from paper_2603_19600_gb300 import _native as nat
    nd, ns, nside = 12, 20000, 64
    o = synth.Observation(nside, synth.satellite_scan(ns, t0=400.0), synth.hex_focal_plane(nd))
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    taps = np.tile(synth.inverse_noise_taps(), (nd, 1))
    N = fx.Noise.banded(P, taps)
    pix, c, s = P.expand(torch.float32)
    taps32 = torch.as_tensor(taps, dtype=torch.float32, device=dev).contiguous()
    bj = fx.blockdiag_precond(P, N)
    valid = bj["valid_u8"]
    g = torch.Generator(device=dev).manual_seed(11)
    xs = [torch.randn(P.npix_total, 3, dtype=torch.float64, device=dev, generator=g) for _ in range(2)]
    for x in xs:
        ref = fx.ptnp_apply(P, N, x, valid, precision="f32", acc="f32")
        out = torch.full_like(x, float("nan"))
        nat.furax_ptnp_apply_noalloc(pix, c, s, nd, ns, nside, taps32, x, out, valid)
        torch.cuda.synchronize()
        # both accumulate FP32 contributions with FP32 atomics in different orders
        err = (torch.linalg.norm(out - ref) / torch.linalg.norm(ref)).item()
        assert err < 1e-5, err
        assert torch.all(out[~bj["valid"]] == 0)


@pytest.mark.parametrize("kind", ["banded", "white"])
@pytest.mark.parametrize("side_stream", [False, True])
def test_noalloc_matches_oracle(fx, dev, orc, kind, side_stream):
    """Against the FP64 oracle on exactly what the kernel reads (the FP32 cache upcast, FP32
    taps or inverse variances that are powers of two, the FP32-rounded map): per element within
    (n_band + n_hits) u of |P^T| |N^-1| |P| |x| (u = 2^-24; plain FP32 accumulation). White noise
    is the one-tap case (ntaps = 1); the side stream is a non-default stream, waited for by the
    current one. Two calls in a row on the shared scratch."""
    from paper_2603_19600_gb300 import _native as nat
    from parity import elem
    nd, ns, nside = 9, 13001, 32
    o = synth.Observation(nside, synth.satellite_scan(ns, t0=700.0), synth.hex_focal_plane(nd))
    P = fx.Pointing.from_observations([o], mode="cache_f32", device=dev)
    pix, c, s = P.cache()
    if kind == "banded":
        taps = np.tile(synth.inverse_noise_taps(), (nd, 1)).astype(np.float32).astype(np.float64)
        on, on_abs = orc.Noise(taps=taps), orc.Noise(taps=np.abs(taps))
    else:
        sig2 = 2.0 ** (3 + np.arange(nd) % 4)
        taps = (1.0 / sig2)[:, None]
        on = on_abs = orc.Noise(sigma2=sig2)
    taps32 = torch.as_tensor(taps, dtype=torch.float32, device=dev).contiguous()
    pts = [a.cpu().numpy().astype(np.float64 if a.dtype == torch.float32 else np.int32).reshape(nd, ns)
           for a in (pix, c, s)]
    g = np.random.default_rng(12)
    valid = g.random(o.npix) > 0.1
    vt = torch.as_tensor(valid.astype(np.uint8), device=dev)
    hits = np.bincount(pts[0][pts[0] >= 0], minlength=o.npix)
    tol = ((129 if kind == "banded" else 2) + int(hits.max()) + 1) * 2.0 ** -24
    st = torch.cuda.Stream(device=dev) if side_stream else torch.cuda.current_stream(dev)
    for rep in range(2):
        x = synth.gaussian_sky(nside, synth.rng(91, rep)).astype(np.float32).astype(np.float64)
        xt = torch.as_tensor(x, device=dev)
        out = torch.full_like(xt, float("nan"))
        st.wait_stream(torch.cuda.current_stream(dev))
        nat.furax_ptnp_apply_noalloc(pix, c, s, nd, ns, nside, taps32, xt, out, vt, stream=st)
        torch.cuda.current_stream(dev).wait_stream(st)
        got = out.cpu().numpy()
        ref = orc.apply_ata(o.npix, *pts, on, valid, x)
        scale = orc.apply_ata(o.npix, pts[0], np.abs(pts[1]), np.abs(pts[2]), on_abs, valid, np.abs(x))
        assert elem(got, ref, scale, f"noalloc {kind} side={side_stream} call {rep}") <= tol
        assert np.all(got[~valid] == 0.0)


def test_noalloc_rejects_maps_above_its_scratch(fx, dev):
    from paper_2603_19600_gb300 import _native as nat
    t = torch.zeros(4, dtype=torch.float32, device=dev)
    p = torch.zeros(4, dtype=torch.int32, device=dev)
    npix = 12 * 512 * 512
    x = torch.zeros(npix, 3, dtype=torch.float64, device=dev)
    with pytest.raises(nat.FuraxError, match="at most"):
        nat.furax_ptnp_apply_noalloc(p, t, t, 1, 4, 512, t[:1], x, torch.zeros_like(x))
