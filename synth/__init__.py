"""Seeded synthetic inputs for map-making: scan, focal plane, sky, noise.

This module produces the *inputs* of the map-making problem only. It holds
none of the method's arithmetic: no quaternion product of the pointing chain,
no pixelisation, no polarisation weights, no projection. Rotations are
composed with ``scipy.spatial.transform.Rotation``. Both the CUDA path and the
FP64 oracle consume the arrays produced here, bit for bit.

Workload recipe (the paper, Statement of Need and Software Design, states the
linear model d = P m + n and the operators but no instrument; the parameters
below are the satellite-like configurations the benchmarks are defined on):

* scan: spin 1 rpm about an axis at 50 deg from the boresight, that axis
  precessing at 45 deg about the anti-sun direction with a 1 h period; the
  anti-sun direction follows the ecliptic over a year; 20 Hz sampling;
* focal plane: co-pointed detectors at given angles, or a hexagonal lattice of
  radius 5 deg with detector angles cycling 0/45/90/135 deg;
* sky: i.i.d. Gaussian I, Q, U per pixel (sigma 100 uK for I, 1 uK for Q, U);
* noise: white (sigma 10 uK) plus 1/f with f_knee 0.1 Hz and slope 1;
* inverse-noise taps: the autocorrelation of 1/PSD, truncated to 64 lags and
  Bartlett-tapered so the banded Toeplitz matrix is positive definite.

Seeds: ``numpy.random.default_rng(20260321 + 100 * config + stream)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.spatial.transform import Rotation

SEED_BASE = 20260321
FSAMP_HZ = 20.0
SIGMA_UK = 10.0
FKNEE_HZ = 0.1
ALPHA = 1.0
NTAPS = 64


def rng(config: int, stream: int) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + 100 * config + stream)


def _wxyz(r: Rotation) -> np.ndarray:
    """Rotation -> quaternion array [..., 4] ordered (w, x, y, z), float64, C-contiguous."""
    q = r.as_quat()  # scipy order (x, y, z, w)
    q = np.atleast_2d(q)
    return np.ascontiguousarray(q[:, [3, 0, 1, 2]], dtype=np.float64)


def satellite_scan(nsamp: int, fsamp: float = FSAMP_HZ, spin_rpm: float = 1.0,
                   opening_deg: float = 50.0, precession_deg: float = 45.0,
                   precession_period_s: float = 3600.0, t0: float = 0.0) -> np.ndarray:
    """Boresight quaternions [nsamp][4] (w, x, y, z) of a spinning, precessing satellite.

    q_b(t) = Rz(lambda_sun(t)) Ry(pi/2) Rz(w_p t) Ry(precession) Rz(w_s t) Ry(opening),
    applied right to left to the boresight axis z.
    """
    t = t0 + np.arange(nsamp, dtype=np.float64) / fsamp
    w_s = 2.0 * math.pi * spin_rpm / 60.0
    w_p = 2.0 * math.pi / precession_period_s
    lam = 2.0 * math.pi * t / (365.25 * 86400.0)
    rz = lambda a: Rotation.from_rotvec(np.outer(np.atleast_1d(a), [0.0, 0.0, 1.0]))
    ry = lambda a: Rotation.from_rotvec(np.outer(np.atleast_1d(a), [0.0, 1.0, 0.0]))
    r = (rz(lam) * ry(math.pi / 2) * rz(w_p * t) * ry(math.radians(precession_deg))
         * rz(w_s * t) * ry(math.radians(opening_deg)))
    return _wxyz(r)


def hwp_angle(nsamp: int, fsamp: float = FSAMP_HZ, hwp_rpm: float = 46.0, t0: float = 0.0,
              omega0: float = 0.0) -> np.ndarray:
    """Angle of a continuously rotating half-wave plate, omega(t) = omega0 + 2 pi (rpm / 60) t."""
    t = t0 + np.arange(nsamp, dtype=np.float64) / fsamp
    return omega0 + 2.0 * math.pi * (hwp_rpm / 60.0) * t


def copointed_detectors(psi_deg) -> np.ndarray:
    """Detectors on the boresight, each rotated by its polarisation angle: q_det = Rz(psi)."""
    psi = np.radians(np.asarray(psi_deg, dtype=np.float64))
    return _wxyz(Rotation.from_rotvec(np.outer(psi, [0.0, 0.0, 1.0])))


def hex_positions(ndet: int):
    """The ndet points of the unit hexagonal lattice nearest the origin.

    Ties in distance are broken by polar angle in [0, 2pi). Returns (radius, angle)
    with the outermost radius scaled to 1 (all zero when ndet == 1).
    """
    k = int(math.ceil(math.sqrt(ndet))) + 2
    pts = []
    for m in range(-k, k + 1):
        for n in range(-k, k + 1):
            r2 = m * m + m * n + n * n  # exact squared radius on the lattice
            x = m + 0.5 * n
            y = n * math.sqrt(3.0) / 2.0
            ang = math.atan2(y, x) % (2.0 * math.pi)
            pts.append((r2, ang, x, y))
    pts.sort(key=lambda p: (p[0], p[1]))
    pts = pts[:ndet]
    rad = np.array([math.sqrt(p[0]) for p in pts])
    ang = np.array([p[1] for p in pts])
    if rad.max() > 0:
        rad = rad / rad.max()
    return rad, ang


def hex_focal_plane(ndet: int, radius_deg: float = 5.0) -> np.ndarray:
    """q_det [ndet][4] on a hexagonal focal plane of the given radius.

    Detector i sits at (rho_i, phi_i) and has polarisation angle 45 deg * (i mod 4):
    q_det = Rz(phi_i) Ry(rho_i) Rz(-phi_i) Rz(psi_i).
    """
    rad, ang = hex_positions(ndet)
    rho = np.radians(radius_deg) * rad
    psi = np.radians(45.0 * (np.arange(ndet) % 4))
    rz = lambda a: Rotation.from_rotvec(np.outer(a, [0.0, 0.0, 1.0]))
    ry = lambda a: Rotation.from_rotvec(np.outer(a, [0.0, 1.0, 0.0]))
    r = rz(ang) * ry(rho) * rz(-ang) * rz(psi)
    return _wxyz(r)


def gaussian_sky(nside: int, g: np.random.Generator, sigma_i: float = 100.0,
                 sigma_qu: float = 1.0) -> np.ndarray:
    """IQU map [12 nside^2][3] float64 with i.i.d. Gaussian pixels (uK)."""
    npix = 12 * nside * nside
    m = np.empty((npix, 3), dtype=np.float64)
    m[:, 0] = g.normal(0.0, sigma_i, npix)
    m[:, 1] = g.normal(0.0, sigma_qu, npix)
    m[:, 2] = g.normal(0.0, sigma_qu, npix)
    return m


def one_over_f_psd(freq: np.ndarray, sigma: float = SIGMA_UK, fknee: float = FKNEE_HZ,
                   alpha: float = ALPHA) -> np.ndarray:
    """PSD(f) = sigma^2 (1 + (fknee/|f|)^alpha) per sample; PSD(0) is returned as +inf."""
    f = np.abs(np.asarray(freq, dtype=np.float64))
    with np.errstate(divide="ignore"):
        return sigma ** 2 * (1.0 + np.where(f > 0, (fknee / np.where(f > 0, f, 1.0)) ** alpha, np.inf))


def inverse_noise_taps(ntaps: int = NTAPS, fsamp: float = FSAMP_HZ, sigma: float = SIGMA_UK,
                       fknee: float = FKNEE_HZ, alpha: float = ALPHA, nfft: int = 1 << 16) -> np.ndarray:
    """Band of the stationary inverse noise covariance, lags 0..ntaps-1 (float64, 1/uK^2).

    c_k = irfft(1/PSD)[k] on an nfft grid (1/PSD(0) taken as its limit 0), then the
    Bartlett taper c_k (1 - k/ntaps), whose symbol is the inverse PSD smoothed by a
    non-negative Fejer kernel, so every finite section is positive definite.
    """
    f = np.fft.rfftfreq(nfft, d=1.0 / fsamp)
    inv = np.zeros_like(f)
    inv[1:] = 1.0 / one_over_f_psd(f[1:], sigma, fknee, alpha)
    c = np.fft.irfft(inv, n=nfft)[:ntaps]
    return c * (1.0 - np.arange(ntaps) / ntaps)


def noise_covariance_band(ntaps: int = NTAPS, fsamp: float = FSAMP_HZ, sigma: float = SIGMA_UK,
                          fknee: float = FKNEE_HZ, alpha: float = ALPHA, fmin: float = 0.01,
                          nfft: int = 1 << 16) -> np.ndarray:
    """Band of a stationary noise covariance, lags 0..ntaps-1 (uK^2): the autocovariance of the
    1/f + white spectrum with the 1/f part cut off below fmin (PSD sigma^2 (1 + (fknee /
    sqrt(f^2 + fmin^2))^alpha)), Bartlett-tapered so that every finite section is positive definite."""
    f = np.fft.rfftfreq(nfft, d=1.0 / fsamp)
    psd = sigma ** 2 * (1.0 + (fknee / np.sqrt(f ** 2 + fmin ** 2)) ** alpha)
    c = np.fft.irfft(psd, n=nfft)[:ntaps]
    return c * (1.0 - np.arange(ntaps) / ntaps)


def band_realization(taps: np.ndarray, nsamp: int, g: np.random.Generator) -> np.ndarray:
    """Gaussian streams [ndet][nsamp] whose covariance is the symmetric band taps [ndet][K]
    (circulant embedding: white noise shaped by the square root of the band's non-negative
    spectrum on a periodic grid longer than nsamp + 2K)."""
    taps = np.atleast_2d(np.asarray(taps, np.float64))
    ndet, k = taps.shape
    n = 1 << int(np.ceil(np.log2(nsamp + 2 * k)))
    kern = np.zeros((ndet, n))
    kern[:, :k] = taps
    kern[:, n - k + 1:] = taps[:, 1:][:, ::-1]
    spec = np.maximum(np.fft.rfft(kern, axis=1).real, 0.0)
    w = g.normal(size=(ndet, n))
    return np.fft.irfft(np.fft.rfft(w, axis=1) * np.sqrt(spec), n=n, axis=1)[:, :nsamp]


def white_noise(ndet: int, nsamp: int, g: np.random.Generator, sigma: float = SIGMA_UK) -> np.ndarray:
    return g.normal(0.0, sigma, (ndet, nsamp))


def one_over_f_noise(ndet: int, nsamp: int, g: np.random.Generator, fsamp: float = FSAMP_HZ,
                     sigma: float = SIGMA_UK, fknee: float = FKNEE_HZ, alpha: float = ALPHA) -> np.ndarray:
    """White + 1/f Gaussian noise [ndet][nsamp], shaped in Fourier space (mean removed)."""
    w = g.normal(0.0, 1.0, (ndet, nsamp))
    f = np.fft.rfftfreq(nsamp, d=1.0 / fsamp)
    psd = one_over_f_psd(f, sigma, fknee, alpha)
    psd[0] = 0.0
    return np.fft.irfft(np.fft.rfft(w, axis=1) * np.sqrt(psd), n=nsamp, axis=1)


@dataclass
class Observation:
    """One observation: boresight, detectors and the pixelisation it is mapped onto."""
    nside: int
    q_bore: np.ndarray           # [nsamp][4] float64 (w, x, y, z)
    q_det: np.ndarray            # [ndet][4] float64
    psi_offset: np.ndarray | None = None  # [ndet] rad
    hwp: np.ndarray | None = None         # [nsamp] half-wave-plate angle (rad) per boresight sample
    map_id: int | None = None             # observations with equal map_id share one map

    @property
    def ndet(self) -> int:
        return self.q_det.shape[0]

    @property
    def nsamp(self) -> int:
        return self.q_bore.shape[0]

    @property
    def npix(self) -> int:
        return 12 * self.nside * self.nside


def config1(nsamp: int = 65536, nside: int = 16):
    """4 co-pointed detectors at 0/45/90/135 deg, white noise, Gaussian sky (plain FP64 case)."""
    obs = Observation(nside, satellite_scan(nsamp), copointed_detectors([0.0, 45.0, 90.0, 135.0]))
    sky = gaussian_sky(nside, rng(1, 0))
    noise = white_noise(obs.ndet, nsamp, rng(1, 1))
    sigma2 = np.full(obs.ndet, SIGMA_UK ** 2)
    return obs, sky, noise, sigma2


def config2(ndet: int = 256, nsamp: int = 1 << 20, nside: int = 512, noise: bool = True):
    """Hex focal plane (radius 5 deg), 1/f + white noise, 64-tap banded inverse noise."""
    obs = Observation(nside, satellite_scan(nsamp), hex_focal_plane(ndet))
    sky = gaussian_sky(nside, rng(2, 0))
    n = one_over_f_noise(ndet, nsamp, rng(2, 1)) if noise else None
    taps = np.tile(inverse_noise_taps(), (ndet, 1))
    return obs, sky, n, taps


def config4_shapes(nobs: int = 64, min_log2: int = 18, max_log2: int = 22, seed_stream: int = 0):
    """Ragged batch shapes: lengths uniform in [2^min, 2^max], 8..128 detectors, nside 256/512 alternating."""
    g = rng(4, seed_stream)
    ns = g.integers(1 << min_log2, (1 << max_log2) + 1, nobs)
    nd = g.integers(8, 129, nobs)
    nside = np.where(np.arange(nobs) % 2 == 0, 256, 512)
    return [(int(nside[i]), int(nd[i]), int(ns[i])) for i in range(nobs)]


def config4(nobs: int = 64, min_log2: int = 18, max_log2: int = 22, nside_override=None):
    """Independent observations, each on its own map; scan segments start at staggered times."""
    shapes = config4_shapes(nobs, min_log2, max_log2)
    out = []
    t0 = 0.0
    for i, (nside, nd, ns) in enumerate(shapes):
        if nside_override is not None:
            nside = nside_override(i, nside)
        obs = Observation(nside, satellite_scan(ns, t0=t0), hex_focal_plane(nd))
        out.append(obs)
        t0 += ns / FSAMP_HZ
    return out


def config5(ndet: int = 128, nsamp: int = 1 << 20, nside: int = 256):
    """Differentiable case: hex focal plane with per-detector angle offsets ~ N(0, 1 deg)."""
    obs = Observation(nside, satellite_scan(nsamp), hex_focal_plane(ndet))
    obs.psi_offset = np.radians(rng(5, 2).normal(0.0, 1.0, ndet))
    sky = gaussian_sky(nside, rng(5, 0))
    taps = np.tile(inverse_noise_taps(), (ndet, 1))
    return obs, sky, taps
