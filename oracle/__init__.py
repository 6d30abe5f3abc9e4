"""FP64 CPU oracle for the map-making hot path — TEST INFRASTRUCTURE.

Plain, slow, obviously correct reference (C, FP64, no FMA contraction) that the
CUDA path is checked against. Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use it. It shares no code with the CUDA library
and imports nothing from it.

Each function follows the paper's operators (Furax, arXiv 2603.19600):
P (PointingOperator, Table 3), P^T (transpose, Table 1), N^-1 (HomothetyOperator /
SymmetricBandToeplitzOperator, Table 2), the block-Jacobi preconditioner
(BJPreconditioner, "Map-making classes"), and the GLS estimator
m = (P^T N^-1 P)^-1 P^T N^-1 d (Statement of Need) solved by PCG (A.I(solver, preconditioner),
Table 1). Conventions the paper leaves open are stated in ``furax_oracle.c``.

Parity status of each function (pins live in ``tests/test_oracle_*.py``):
  quat_mul, quat_axes      pinned (scipy rotations, orthonormality)
  phi                      pinned (libm atan2 within 4 ulp, exact special angles)
  ang2pix / pix2ang        pinned (closed forms, round trips, projection-plane lookup,
                           equal-area counts, ring structure)
  pointing weights         pinned (angle rotation about the line of sight, c^2+s^2=1,
                           closed form for co-pointed detectors)
  P, P^T, hits             pinned (adjoint identity, bincount, dense matrix)
  ninv_white / ninv_band   pinned (dense Toeplitz, FFT circular embedding, symmetry, SPD)
  bj / bj_apply            pinned (closed form diag(4,2,2)/sigma^2, numpy inverse, SPD)
  rhs / apply_ata / pcg    pinned (dense normal equations at nside 1-2, one-step
                           convergence for white noise, noiseless recovery)
  chi2_grad                pinned (central finite differences)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "furax_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (host architecture, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_P = ctypes.c_void_p
_I = ctypes.c_int64
_D = ctypes.c_double

_SIGS = {
    "orc_phi": (_D, [_D, _D]),
    "orc_ang2pix_ring": (_I, [_I, _D, _D]),
    "orc_ang2pix_ring_batch": (None, [_I, _I, _P, _P, _P]),
    "orc_vec2pix_ring_batch": (None, [_I, _I, _P, _P]),
    "orc_pix2ang_ring_batch": (None, [_I, _I, _P, _P, _P]),
    "orc_phi_batch": (None, [_I, _P, _P, _P]),
    "orc_quat_mul_batch": (None, [_I, _P, _P, _P]),
    "orc_quat_axes_batch": (None, [_I, _P, _P, _P]),
    "orc_pointing": (_I, [_I, _I, _P, _I, _P, _P, _P, _P, _P, _P]),
    "orc_P": (None, [_I, _P, _P, _P, _P, _P]),
    "orc_PT": (None, [_I, _I, _P, _P, _P, _P, _P, _P]),
    "orc_ninv_white": (None, [_I, _I, _P, _P, _P]),
    "orc_ninv_band": (None, [_I, _I, _I, _P, _P, _P]),
    "orc_bj": (None, [_I, _I, _I, _P, _P, _P, _P, _D, _P, _P, _P, _P, _P]),
    "orc_bj_apply": (None, [_I, _P, _P, _P, _P]),
    "orc_rhs": (None, [_I, _I, _I, _P, _P, _P, ctypes.c_int, _P, _P, _I, _P, _P, _P]),
    "orc_apply_ata": (None, [_I, _I, _I, _P, _P, _P, ctypes.c_int, _P, _P, _I, _P, _P, _P]),
    "orc_pcg": (_I, [_I, _I, _I, _P, _P, _P, ctypes.c_int, _P, _P, _I, _P, _P, _P, _P, _I, _D, _P]),
    "orc_chi2_grad": (_D, [_I, _I, _I, _P, _P, _P, ctypes.c_int, _P, _P, _I, _P, _P, _P, _P]),
}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = ctypes.CDLL(build())
            for name, (res, args) in _SIGS.items():
                f = getattr(l, name)
                f.restype = res
                f.argtypes = args
            _lib = l
    return _lib


def _c(a, dtype):
    """Contiguous array of the exact dtype; raises instead of silently converting widths."""
    a = np.ascontiguousarray(a)
    if a.dtype != dtype:
        a = np.ascontiguousarray(a, dtype=dtype)
    return a


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- geometry
def quat_mul(a, b):
    a = _c(np.atleast_2d(a), np.float64); b = _c(np.atleast_2d(b), np.float64)
    a, b = np.broadcast_arrays(a, b); a = _c(a, np.float64); b = _c(b, np.float64)
    out = np.empty_like(a)
    lib().orc_quat_mul_batch(a.shape[0], _p(a), _p(b), _p(out))
    return out


def quat_axes(q):
    q = _c(np.atleast_2d(q), np.float64)
    d = np.empty((q.shape[0], 3)); o = np.empty((q.shape[0], 3))
    lib().orc_quat_axes_batch(q.shape[0], _p(q), _p(d), _p(o))
    return d, o


def phi(x, y):
    x = _c(np.atleast_1d(x), np.float64); y = _c(np.atleast_1d(y), np.float64)
    out = np.empty_like(x)
    lib().orc_phi_batch(x.size, _p(x), _p(y), _p(out))
    return out


def ang2pix(nside, z, phi_):
    z = _c(np.atleast_1d(z), np.float64); phi_ = _c(np.atleast_1d(phi_), np.float64)
    out = np.empty(z.shape, np.int64)
    lib().orc_ang2pix_ring_batch(nside, z.size, _p(z), _p(phi_), _p(out))
    return out


def vec2pix(nside, v):
    v = _c(np.atleast_2d(v), np.float64)
    out = np.empty(v.shape[0], np.int64)
    lib().orc_vec2pix_ring_batch(nside, v.shape[0], _p(v), _p(out))
    return out


def pix2ang(nside, pix):
    pix = _c(np.atleast_1d(pix), np.int64)
    z = np.empty(pix.shape); ph = np.empty(pix.shape)
    lib().orc_pix2ang_ring_batch(nside, pix.size, _p(pix), _p(z), _p(ph))
    return z, ph


# ---------------------------------------------------------------- pointing
def pointing(nside, q_bore, q_det, psi_offset=None, hwp=None):
    """Per-sample RING pixel (int32) and weights cos 2psi, sin 2psi (float64), each [ndet][nsamp].
    With hwp (angle per boresight sample) the weights are cos(4 hwp - 2psi), sin(4 hwp - 2psi)."""
    qb = _c(q_bore, np.float64); qd = _c(q_det, np.float64)
    ns, nd = qb.shape[0], qd.shape[0]
    po = None if psi_offset is None else _c(psi_offset, np.float64)
    hw = None if hwp is None else _c(hwp, np.float64)
    assert hw is None or hw.shape == (ns,)
    pix = np.empty((nd, ns), np.int32); c = np.empty((nd, ns)); s = np.empty((nd, ns))
    bad = lib().orc_pointing(nside, ns, _p(qb), nd, _p(qd), _p(po), _p(hw), _p(pix), _p(c), _p(s))
    return pix, c, s, int(bad)


def P(pix, c, s, m):
    pix = _c(pix, np.int32); c = _c(c, np.float64); s = _c(s, np.float64); m = _c(m, np.float64)
    tod = np.empty(pix.shape)
    lib().orc_P(pix.size, _p(pix), _p(c), _p(s), _p(m), _p(tod))
    return tod


def PT(npix, pix, c, s, tod):
    pix = _c(pix, np.int32); c = _c(c, np.float64); s = _c(s, np.float64); tod = _c(tod, np.float64)
    m = np.empty((npix, 3)); hits = np.empty(npix, np.int32)
    lib().orc_PT(npix, pix.size, _p(pix), _p(c), _p(s), _p(tod), _p(m), _p(hits))
    return m, hits


# ---------------------------------------------------------------- noise
def ninv_white(sigma2, x):
    x = _c(x, np.float64); sigma2 = _c(sigma2, np.float64)
    y = np.empty_like(x)
    lib().orc_ninv_white(x.shape[0], x.shape[1], _p(sigma2), _p(x), _p(y))
    return y


def ninv_band(taps, x):
    x = _c(x, np.float64); taps = _c(np.atleast_2d(taps), np.float64)
    y = np.empty_like(x)
    lib().orc_ninv_band(x.shape[0], x.shape[1], taps.shape[1], _p(taps), _p(x), _p(y))
    return y


# ---------------------------------------------------------------- preconditioner and solver
class Noise:
    """White noise (sigma2 [ndet]) or banded inverse covariance (taps [ndet][K])."""

    def __init__(self, sigma2=None, taps=None):
        assert (sigma2 is None) != (taps is None)
        self.kind = 0 if sigma2 is not None else 1
        self.sigma2 = None if sigma2 is None else _c(sigma2, np.float64)
        self.taps = None if taps is None else _c(np.atleast_2d(taps), np.float64)

    @property
    def ntaps(self):
        return 0 if self.taps is None else self.taps.shape[1]

    def diag(self):
        return 1.0 / self.sigma2 if self.kind == 0 else self.taps[:, 0].copy()

    def apply(self, x):
        return ninv_white(self.sigma2, x) if self.kind == 0 else ninv_band(self.taps, x)


def bj(npix, pix, c, s, noise: Noise, rcond_min=1e-3):
    pix = _c(pix, np.int32); c = _c(c, np.float64); s = _c(s, np.float64)
    nd, ns = pix.shape
    diag = _c(noise.diag(), np.float64)
    blocks = np.empty((npix, 6)); inv = np.empty((npix, 6)); valid = np.empty(npix, np.uint8)
    hits = np.empty(npix, np.int32); rcond = np.empty(npix)
    lib().orc_bj(npix, nd, ns, _p(pix), _p(c), _p(s), _p(diag), rcond_min,
                 _p(blocks), _p(inv), _p(valid), _p(hits), _p(rcond))
    return dict(blocks=blocks, inv=inv, valid=valid.astype(bool), hits=hits, rcond=rcond)


def bj_apply(inv, valid, r):
    inv = _c(inv, np.float64); r = _c(r, np.float64); v = _c(valid, np.uint8)
    z = np.empty_like(r)
    lib().orc_bj_apply(inv.shape[0], _p(inv), _p(v), _p(r), _p(z))
    return z


def _noise_args(noise: Noise):
    return (noise.kind, _p(noise.sigma2), _p(noise.taps), noise.ntaps)


def rhs(npix, pix, c, s, noise: Noise, valid, d):
    pix = _c(pix, np.int32); c = _c(c, np.float64); s = _c(s, np.float64); d = _c(d, np.float64)
    v = None if valid is None else _c(valid, np.uint8)
    out = np.empty((npix, 3))
    lib().orc_rhs(npix, pix.shape[0], pix.shape[1], _p(pix), _p(c), _p(s), *_noise_args(noise),
                  _p(v), _p(d), _p(out))
    return out


def apply_ata(npix, pix, c, s, noise: Noise, valid, x):
    pix = _c(pix, np.int32); c = _c(c, np.float64); s = _c(s, np.float64); x = _c(x, np.float64)
    v = None if valid is None else _c(valid, np.uint8)
    out = np.empty((npix, 3))
    lib().orc_apply_ata(npix, pix.shape[0], pix.shape[1], _p(pix), _p(c), _p(s), *_noise_args(noise),
                        _p(v), _p(x), _p(out))
    return out


def pcg(npix, pix, c, s, noise: Noise, valid, minv, b, maxiter, tol=1e-8):
    pix = _c(pix, np.int32); c = _c(c, np.float64); s = _c(s, np.float64); b = _c(b, np.float64)
    v = _c(valid, np.uint8); minv = _c(minv, np.float64)
    x = np.empty((npix, 3)); hist = np.zeros(maxiter + 1)
    it = lib().orc_pcg(npix, pix.shape[0], pix.shape[1], _p(pix), _p(c), _p(s), *_noise_args(noise),
                       _p(v), _p(minv), _p(b), _p(x), maxiter, tol, _p(hist))
    return x, int(it), hist[: it + 1]


def chi2_grad(npix, pix, c, s, noise: Noise, m, d, want_grad=True, hwp=False):
    """chi^2 and its gradients. With an ideal half-wave plate (hwp=True) the weights are
    cos(4w - 2psi - 2delta), sin(...): their derivative in delta is minus the one without it."""
    pix = _c(pix, np.int32); c = _c(c, np.float64); s = _c(s, np.float64)
    m = _c(m, np.float64); d = _c(d, np.float64)
    gm = np.empty((npix, 3)) if want_grad else None
    gp = np.empty(pix.shape[0]) if want_grad else None
    chi2 = lib().orc_chi2_grad(npix, pix.shape[0], pix.shape[1], _p(pix), _p(c), _p(s),
                               *_noise_args(noise), _p(m), _p(d), _p(gm), _p(gp))
    if want_grad and hwp:
        gp = -gp
    return chi2, gm, gp


def binned_map(bjd, b):
    """m_p = M_p^-1 b_p on valid pixels (the binned estimator), 0 elsewhere."""
    return bj_apply(bjd["inv"], bjd["valid"], b)
