"""The encoding-level FP32 <-> FP64 conversions (used where FP64 conversion instructions would
occupy the FP64 pipe) against the IEEE 754 conversions of numpy and of the GPU, bit for bit:
round-to-nearest-even ties with odd and even kept parts, the overflow tie above FLT_MAX, both
sides of the binary32 normal range, signed zeros, infinities, NaNs and a few million random
encodings."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _f64_cases(g):
    m = g.integers(1 << 23, 1 << 24, 4096, dtype=np.uint64)      # 24-bit significands, odd and even
    e = g.integers(-120, 120, 4096)
    base = np.ldexp(m.astype(np.float64), e - 23)                  # exactly representable in binary32
    ulp = np.ldexp(1.0, e - 23)
    ties = np.concatenate([base + ulp / 2, -(base + ulp / 2), base - ulp / 2])   # exact ties (both parities)
    near = np.concatenate([base + ulp / 2 * (1 + 2.0 ** -28), base + ulp / 2 * (1 - 2.0 ** -28)])
    fmax = float(np.finfo(np.float32).max)
    edge = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, fmax, -fmax,
                     fmax + np.ldexp(1.0, 103), -(fmax + np.ldexp(1.0, 103)),          # overflow ties
                     fmax + np.ldexp(1.0, 103) * (1 - 2.0 ** -20), np.ldexp(1.0, 128),
                     np.ldexp(1.0, -126), np.ldexp(1.0, -126) * (1 + 2.0 ** -30), np.ldexp(1.0, -126) * (1 - 2.0 ** -30),
                     np.ldexp(1.0, -127), np.ldexp(1.0, -149), np.ldexp(1.0, -150), np.ldexp(1.0, -151),
                     np.ldexp(1.5, -150), 5e-324, -5e-324, 1.0, -1.0, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24])
    rnd = g.integers(0, 2 ** 63, 3_000_000, dtype=np.int64).view(np.float64)     # random encodings
    rnd = np.concatenate([rnd, -rnd])
    return np.concatenate([ties, near, edge, rnd])


def _same_bits32(a, b):
    both_nan = np.isnan(a) & np.isnan(b)
    return np.array_equal(a.view(np.uint32)[~both_nan], b.view(np.uint32)[~both_nan]) and np.array_equal(
        np.isnan(a), np.isnan(b))


def _same_bits64(a, b):
    both_nan = np.isnan(a) & np.isnan(b)
    return np.array_equal(a.view(np.uint64)[~both_nan], b.view(np.uint64)[~both_nan]) and np.array_equal(
        np.isnan(a), np.isnan(b))


def test_f64_to_f32_is_round_to_nearest_even(fx, dev):
    from paper_2603_19600_gb300 import _native as nat
    v = _f64_cases(np.random.default_rng(1))
    vt = torch.as_tensor(v, device=dev)
    out = torch.empty(v.size, dtype=torch.float32, device=dev)
    with np.errstate(over="ignore"):
        ref_np = v.astype(np.float32)
    nat.furax_probe_convert(in64=vt, out32=out)
    got = out.cpu().numpy()
    assert _same_bits32(got, ref_np)
    assert _same_bits32(got, vt.float().cpu().numpy())          # the GPU's own conversion


def test_f32_to_f64_is_exact(fx, dev):
    from paper_2603_19600_gb300 import _native as nat
    g = np.random.default_rng(2)
    f = np.concatenate([g.integers(0, 2 ** 32, 3_000_000, dtype=np.uint64).astype(np.uint32).view(np.float32),
                        np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 1.17549435e-38,
                                  float(np.finfo(np.float32).max)], dtype=np.float32)])
    ft = torch.as_tensor(f, device=dev)
    out = torch.empty(f.size, dtype=torch.float64, device=dev)
    nat.furax_probe_convert(in32=ft, out64=out)
    got = out.cpu().numpy()
    assert _same_bits64(got, f.astype(np.float64))
    assert _same_bits64(got, ft.double().cpu().numpy())
