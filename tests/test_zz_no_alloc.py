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


def test_noalloc_rejects_maps_above_its_scratch(fx, dev):
    from paper_2603_19600_gb300 import _native as nat
    t = torch.zeros(4, dtype=torch.float32, device=dev)
    p = torch.zeros(4, dtype=torch.int32, device=dev)
    npix = 12 * 512 * 512
    x = torch.zeros(npix, 3, dtype=torch.float64, device=dev)
    with pytest.raises(nat.FuraxError, match="at most"):
        nat.furax_ptnp_apply_noalloc(p, t, t, 1, 4, 512, t[:1], x, torch.zeros_like(x))
