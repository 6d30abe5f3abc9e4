"""Map-making on GB300: pointing P, noise weighting N^-1, block-Jacobi, PCG, chi^2 gradients.

Thin object layer over the C ABI (``_native``): it allocates outputs with torch and
passes pointers; every computation runs in libfurax's CUDA kernels. Names follow the
paper's operators (Furax, arXiv 2603.19600): PointingOperator (P), its transpose,
HomothetyOperator / SymmetricBandToeplitzOperator (N^-1), BJPreconditioner, and the
maximum-likelihood estimator (P^T N^-1 P)^-1 P^T N^-1 d solved by PCG.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
from dataclasses import dataclass, field

import torch

from . import _native as nat

_MODES = {"on_the_fly": nat.FURAX_POINTING_ON_THE_FLY, "cache_f32": nat.FURAX_POINTING_CACHE_F32,
          "cache_f64": nat.FURAX_POINTING_CACHE_F64, "cache_mixed": nat.FURAX_POINTING_CACHE_MIXED}
_ACC = {"f64": nat.FURAX_ACC_F64, "f32_kahan": nat.FURAX_ACC_F32_KAHAN, "f32": nat.FURAX_ACC_F32}
_PREC = {"f32": nat.FURAX_F32, "f64": nat.FURAX_F64, "f32x2": nat.FURAX_PREC_F32X2}


class Pointing:
    """Pointing operator of a batch of observations (one map per observation).

    q_bore: float64 [sum nsamp][4] (w, x, y, z); q_det: float64 [sum ndet][4]; both on the GPU
    and kept alive by this object. mode: "cache_f32" (pixel + FP32 weights cached, 12 B/sample),
    "cache_f64" (20 B/sample) or "on_the_fly" (recomputed from the quaternions each call).
    hwp_angle: optional float64 [sum nsamp] angle of an ideal half-wave plate per boresight sample
    (weights become cos(4w - 2psi), sin(4w - 2psi)); read once here.
    """

    def __init__(self, q_bore, q_det, ndet, nsamp, nside, psi_offset=None, mode="cache_f32", stream=None,
                 hwp_angle=None, map_id=None):
        self.ndet, self.nsamp, self.nside = [list(map(int, v)) for v in (ndet, nsamp, nside)]
        self.q_bore = q_bore.contiguous()
        self.q_det = q_det.contiguous()
        self.mode = mode
        self.handle = None
        self.has_hwp = hwp_angle is not None
        self.map_id = None if map_id is None else [int(v) for v in map_id]
        self.handle = nat.furax_pointing_create(self.q_bore, self.q_det, self.ndet, self.nsamp, self.nside,
                                                psi_offset, _MODES[mode], stream,
                                                None if hwp_angle is None else hwp_angle.contiguous(), self.map_id)
        info = nat.furax_pointing_info(self.handle)
        self.nsamp_total = info["nsamp_total"]
        self.npix_total = info["npix_total"]
        self.ndet_total = info["ndet_total"]
        self.n_invalid = info["n_invalid"]
        self.device = self.q_bore.device

    @classmethod
    def from_observations(cls, observations, mode="cache_f32", device="cuda", stream=None):
        """Build from objects with .q_bore, .q_det (numpy) and .nside (see the synth module)."""
        qb = torch.cat([torch.as_tensor(o.q_bore) for o in observations]).to(device, torch.float64)
        qd = torch.cat([torch.as_tensor(o.q_det) for o in observations]).to(device, torch.float64)
        psi = None
        if any(getattr(o, "psi_offset", None) is not None for o in observations):
            psi = torch.cat([torch.as_tensor(o.psi_offset if o.psi_offset is not None else [0.0] * o.ndet)
                             for o in observations]).to(device, torch.float64)
        hw = [getattr(o, "hwp", None) for o in observations]
        if any(h is not None for h in hw) and any(h is None for h in hw):
            raise ValueError("either every observation has a half-wave plate angle stream or none has")
        hwp = None
        if hw[0] is not None:
            hwp = torch.cat([torch.as_tensor(h) for h in hw]).to(device, torch.float64)
        ids = [getattr(o, "map_id", None) for o in observations]
        map_id = None
        if any(m is not None for m in ids):
            # an observation without a map_id keeps a map of its own
            used = {m for m in ids if m is not None}
            fresh = iter(k for k in range(-1, -10 ** 9, -1) if k not in used)
            map_id = [m if m is not None else next(fresh) for m in ids]
        return cls(qb, qd, [o.q_det.shape[0] for o in observations], [o.q_bore.shape[0] for o in observations],
                   [o.nside for o in observations], psi, mode, stream, hwp, map_id)

    def close(self):
        if self.handle:
            nat.furax_pointing_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_schedule(self, kernel="time_ordered", tile_len=0, max_rows=12, group_tol=2.0, l2_evict_first=0,
                     consumer_warps=0):
        """How the cached FP32 normal operator walks the samples: "time_ordered" (one detector x
        4096 samples per tile) or "pixel_sorted" (detectors on one track x tile_len samples, samples
        sorted by pixel once per refresh; see furax_schedule); l2_evict_first=1 reads the pointing
        stream with an L2 evict-first policy; consumer_warps (8 or 16, time-ordered kernel) sets how many
        warps run the band and the scatter. Only the order of the floating-point additions changes."""
        k = {"time_ordered": nat.FURAX_SCHED_TIME_ORDERED, "pixel_sorted": nat.FURAX_SCHED_PIXEL_SORTED}[kernel]
        nat.furax_pointing_set_schedule(self.handle, k, tile_len, max_rows, group_tol, l2_evict_first, consumer_warps)

    def schedule(self) -> dict:
        s = nat.furax_pointing_get_schedule(self.handle)
        s["kernel"] = "pixel_sorted" if s["kernel"] == nat.FURAX_SCHED_PIXEL_SORTED else "time_ordered"
        return s

    def refresh(self):
        """Recompute the cached pointing from the (possibly updated) quaternion tensors."""
        nat.furax_pointing_refresh(self.handle)

    def set_psi_offset(self, psi_offset):
        nat.furax_pointing_set_psi_offset(self.handle, None if psi_offset is None else psi_offset.contiguous())

    def expand(self, dtype=torch.float64):
        """Per-sample pixel (int32, local to its observation) and weights cos 2psi, sin 2psi."""
        pix = torch.empty(self.nsamp_total, dtype=torch.int32, device=self.device)
        c = torch.empty(self.nsamp_total, dtype=dtype, device=self.device)
        s = torch.empty_like(c)
        nat.furax_pointing_expand(self.handle, pix, c, s)
        return pix, c, s

    def cache(self):
        """Pixels and FP32 weights as cached for the FP32 operators (FP32 or mixed cache modes)."""
        pix = torch.empty(self.nsamp_total, dtype=torch.int32, device=self.device)
        c = torch.empty(self.nsamp_total, dtype=torch.float32, device=self.device)
        s = torch.empty_like(c)
        nat.furax_pointing_cache(self.handle, pix, c, s)
        return pix, c, s

    def apply(self, m, out=None, dtype=None):
        """tod = P m; m: [npix_total][3]."""
        if out is None:
            out = torch.empty(self.nsamp_total, dtype=dtype or m.dtype, device=self.device)
        nat.furax_pointing_apply(self.handle, m.contiguous(), out)
        return out

    def transpose(self, tod, out=None, acc="f64", hits=False, dtype=torch.float64, accumulate=False):
        """map = P^T tod (and hit counts when hits=True)."""
        if out is None:
            out = torch.zeros(self.npix_total, 3, dtype=dtype, device=self.device)
        h = torch.zeros(self.npix_total, dtype=torch.int32, device=self.device) if hits else None
        nat.furax_pointing_transpose(self.handle, tod.contiguous(), out, _ACC[acc], h, accumulate)
        return (out, h) if hits else out


class Noise:
    """Inverse noise covariance per detector: white (variances) or a symmetric band (taps)."""

    def __init__(self, pointing: Pointing, kind: str, params: torch.Tensor, stream=None):
        self.kind = kind
        p = params.to(pointing.device, torch.float64).contiguous()
        if kind == "white":
            self.ntaps = 1
            h = nat.furax_noise_create(nat.FURAX_NOISE_WHITE, p.reshape(-1), 1, pointing.ndet, pointing.nsamp,
                                       pointing.nside, stream)
        elif kind == "banded":
            p = p.reshape(pointing.ndet_total, -1)
            self.ntaps = p.shape[1]
            h = nat.furax_noise_create(nat.FURAX_NOISE_BANDED, p, self.ntaps, pointing.ndet, pointing.nsamp,
                                       pointing.nside, stream)
        else:
            raise ValueError(f"unknown noise kind {kind}")
        self.handle = h
        self.params = p

    @classmethod
    def white(cls, pointing, sigma2):
        return cls(pointing, "white", torch.as_tensor(sigma2))

    @classmethod
    def banded(cls, pointing, taps):
        return cls(pointing, "banded", torch.as_tensor(taps))

    def close(self):
        if self.handle:
            nat.furax_noise_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def inv_apply(self, x, out=None):
        if out is None:
            out = torch.empty_like(x)
        nat.furax_noise_inv_apply(self.handle, x.contiguous(), out)
        return out


class Templates:
    """Template deprojection F_T = W - W T (T^T W T)^-1 T^T W with W = N^-1 and, per detector, the
    Legendre polynomials P_0..P_order (order <= 3) of the scaled time 2t/(ns-1) - 1."""

    def __init__(self, pointing: Pointing, noise: Noise, order: int, stream=None):
        self.pointing, self.noise, self.order = pointing, noise, int(order)
        self.handle = None
        self.handle = nat.furax_templates_create(pointing.handle, noise.handle, self.order, stream)

    def close(self):
        if self.handle:
            nat.furax_templates_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def gram(self):
        """T^T W T per detector: float64 [ndet_total][order+1][order+1]."""
        k = self.order + 1
        g = torch.empty(self.pointing.ndet_total, k, k, dtype=torch.float64, device=self.pointing.device)
        nat.furax_templates_gram(self.handle, g)
        return g

    def deproject(self, tod, out=None):
        """F_T tod over the whole TOD (float32 or float64 [nsamp_total])."""
        out = torch.empty_like(tod) if out is None else out
        nat.furax_deproject_apply(self.handle, tod.contiguous(), out)
        return out


def gapfill(cov: Noise, d, valid, n_real, maxiter=1000, tol=1e-10, out=None, precision="f64"):
    """Fill the gaps (valid == 0) of the TOD d with the constrained realisation
    n_g + N_gv N_vv^-1 (d_v - n_v); cov is a banded Noise whose taps hold the covariance band N,
    n_real a realisation of covariance N; precision "f32" applies N in FP32, "f32x2" FP64-accurate
    in double-FP32 on the FP32 units (bands of up to 64 taps), "f64" in FP64. The TOD-sized
    workspaces stay in cov for later calls. Returns (filled TOD, per-detector iterations,
    converged)."""
    if cov.kind != "banded":
        raise ValueError("the covariance must be a banded noise model")
    out = torch.empty_like(d) if out is None else out
    rc, iters = nat.furax_gapfill(cov.handle, cov.params.shape[0], d.contiguous(), valid.to(torch.uint8).contiguous(),
                                  n_real.contiguous(), out, maxiter, tol, _PREC[precision])
    return out, iters, rc == nat.FURAX_OK


def ptfp_apply(T: Templates, x, valid=None, precision="f32", acc="f32", out=None):
    """out = S P^T F_T P S^T x (x float64 [npix_total][3])."""
    if out is None:
        out = torch.empty_like(x)
    v = None if valid is None else valid.to(torch.uint8).contiguous()
    nat.furax_ptfp_apply(T.handle, x.contiguous(), out, v, _PREC[precision], _ACC[acc])
    return out


def blockdiag_precond(P: Pointing, N: Noise, rcond_min=1e-3):
    inv = torch.empty(P.npix_total, 6, dtype=torch.float64, device=P.device)
    valid = torch.empty(P.npix_total, dtype=torch.uint8, device=P.device)
    hits = torch.empty(P.npix_total, dtype=torch.int32, device=P.device)
    rcond = torch.empty(P.npix_total, dtype=torch.float64, device=P.device)
    nat.furax_blockdiag_precond(P.handle, N.handle, rcond_min, inv, valid, hits, rcond)
    return dict(inv=inv, valid=valid.bool(), valid_u8=valid, hits=hits, rcond=rcond)


def ptnp_apply(P: Pointing, N: Noise, x, valid=None, precision="f32", acc="f32", out=None):
    """out = S P^T N^-1 P S^T x (x float64 [npix_total][3])."""
    if out is None:
        out = torch.empty_like(x)
    v = None if valid is None else valid.to(torch.uint8).contiguous()
    nat.furax_ptnp_apply(P.handle, N.handle, x.contiguous(), out, v, _PREC[precision], _ACC[acc])
    return out


def rhs(P: Pointing, N: Noise, d, valid=None):
    b = torch.empty(P.npix_total, 3, dtype=torch.float64, device=P.device)
    v = None if valid is None else valid.to(torch.uint8).contiguous()
    nat.furax_rhs(P.handle, N.handle, d.contiguous(), b, v)
    return b


@dataclass
class SolveInfo:
    status: int
    iters: int
    outer: int
    rel_res: float
    true_rel_res: float
    n_valid: int
    history: list = field(default_factory=list)

    @property
    def converged(self) -> bool:
        return self.status == nat.FURAX_OK


def mapmaker_cg(P: Pointing, N: Noise, d, maxiter=50, tol=1e-8, precision="f64", acc="f32", inner_tol=1e-5,
                max_outer=8, use_graph=True, check_every=10, rcond_min=1e-3, binned_only=False, hist_len=None,
                out=None, true_residual=True, templates: "Templates | None" = None, amplitudes=None,
                d_ready=None, allreduce=None):
    """Solve the map-making normal equations per observation; returns (map, valid mask, SolveInfo).
    With ``templates`` the system is the deprojected one (P^T F_T P) x = P^T F_T d; ``amplitudes``
    (float64 [ndet_total][order+1], optional) then receives the template amplitudes of the map.
    ``d_ready`` (a torch.cuda.Event recorded once d is written) lets the solver start its
    preconditioner before d has arrived. ``allreduce`` (detector sharding: this process holds a
    subset of the detectors of every observation) is fn(tensor), summing a CUDA tensor in place over
    the processes, e.g. ``torch.distributed.all_reduce``; every process calls mapmaker_cg with the
    same layout and gets the same map."""
    o = nat.default_cg_opts()
    o.maxiter, o.tol, o.precision, o.acc = int(maxiter), float(tol), _PREC[precision], _ACC[acc]
    o.inner_tol, o.max_outer, o.use_graph = float(inner_tol), int(max_outer), int(bool(use_graph))
    o.check_every, o.rcond_min, o.binned_only = int(check_every), float(rcond_min), int(bool(binned_only))
    o.true_residual = int(bool(true_residual))
    o.d_ready = None if d_ready is None else d_ready.cuda_event
    cb = None
    if allreduce is not None:
        cb = nat.allreduce_callback(allreduce)
        o.allreduce = ctypes.cast(cb, ctypes.c_void_p)
    x = out if out is not None else torch.empty(P.npix_total, 3, dtype=torch.float64, device=P.device)
    valid = torch.empty(P.npix_total, dtype=torch.uint8, device=P.device)
    hl = hist_len if hist_len is not None else maxiter + 1
    if templates is not None:
        if templates.pointing is not P or templates.noise is not N:
            raise ValueError("templates were built for another pointing or noise")
        rc, res, hist = nat.furax_mapmaker_cg_deproject(templates.handle, d.contiguous(), x, valid, o, hl, amplitudes)
    else:
        rc, res, hist = nat.furax_mapmaker_cg(P.handle, N.handle, d.contiguous(), x, valid, o, hl)
    del cb
    return x, valid.bool(), SolveInfo(rc, res.iters, res.outer, res.rel_res, res.true_rel_res, res.n_valid, hist)


def chi2_grad(P: Pointing, N: Noise, d, m, precision="f64", want_map=True, want_psi=True):
    """chi^2 per observation, d chi^2/d m [npix_total][3] and d chi^2/d psi_det [ndet_total]."""
    chi2 = torch.empty(len(P.ndet), dtype=torch.float64, device=P.device)
    gm = torch.empty(P.npix_total, 3, dtype=torch.float64, device=P.device) if want_map else None
    gp = torch.empty(P.ndet_total, dtype=torch.float64, device=P.device) if want_psi else None
    nat.furax_chi2_grad(P.handle, N.handle, d.contiguous(), m.contiguous(), chi2, gm, gp, _PREC[precision])
    return chi2, gm, gp


class Chi2(torch.autograd.Function):
    """chi^2(m, delta) = (d - P(delta) m)^T N^-1 (d - P(delta) m), summed over observations.

    forward(m, psi_offset, P, N, d, precision) -> scalar; the backward is the hand-written
    gradient pair d chi^2/d m = -2 P^T N^-1 r and d chi^2/d delta_j = -2 sum_t (N^-1 r) 2 (U c - Q s),
    computed by one fused kernel in the forward pass and scaled by the incoming gradient.
    """

    @staticmethod
    def forward(ctx, m, psi_offset, P: Pointing, N: Noise, d, precision="f64"):
        P.set_psi_offset(psi_offset.detach().to(torch.float64).contiguous())
        chi2, gm, gp = chi2_grad(P, N, d, m.detach().to(torch.float64), precision,
                                 want_map=ctx.needs_input_grad[0], want_psi=ctx.needs_input_grad[1])
        ctx.save_for_backward(*(t for t in (gm, gp) if t is not None))
        ctx.has = (gm is not None, gp is not None)
        return chi2.sum().to(m.dtype)

    @staticmethod
    def backward(ctx, g):
        saved = list(ctx.saved_tensors)
        gm = saved.pop(0) * g if ctx.has[0] else None
        gp = saved.pop(0) * g if ctx.has[1] else None
        return gm, gp, None, None, None, None


def chi2(m, psi_offset, P: Pointing, N: Noise, d, precision="f64"):
    return Chi2.apply(m, psi_offset, P, N, d, precision)


_KERNELS = {0: "time_ordered", 1: "pixel_sorted"}


def _tune_key(P: Pointing, N: "Noise", acc: str) -> str:
    """Cache key of a tuned schedule: GPU, pixelisations, detectors, samples (power-of-two bucket),
    pointing mode, noise kind and accumulation."""
    name = torch.cuda.get_device_name(P.device)
    bucket = int(round(math.log2(max(P.nsamp_total, 1))))
    nsides = "/".join(str(n) for n in sorted(set(P.nside)))
    return f"{name}|nside={nsides}|ndet={P.ndet_total}|nsamp=2^{bucket}|{P.mode}|{N.kind}|{acc}"


def default_tune_cache() -> str:
    return os.environ.get("FURAX_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "furax_gb300", "schedules.json"))


def autotune(P: Pointing, N: "Noise", acc: str = "f32_kahan", reps: int = 3, cache_path: str | None = None,
             candidates: list | None = None, retune: bool = False) -> dict:
    """Pick the fastest schedule of the cached FP32 normal operator for this workload and set it on P.

    The search (furax_autotune: each candidate timed on the GPU with CUDA events) runs once per key
    of ``_tune_key``; the result is stored in a JSON file (``cache_path``, default
    ``$FURAX_TUNE_CACHE`` or ``~/.cache/furax_gb300/schedules.json``) and later calls with the same
    key set the stored schedule without timing. The accumulation mode is part of the key and is
    never changed. Returns {"schedule", "ms", "cached", "key", "candidates_timed"}."""
    path = cache_path or default_tune_cache()
    key = _tune_key(P, N, acc)
    table = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
    if not retune and key in table:
        sch = table[key]["schedule"]
        P.set_schedule(sch["kernel"], sch["tile_len"], sch["max_rows"], sch["group_tol"], sch.get("l2_evict_first", 0),
                       sch.get("consumer_warps", 0))
        return {**table[key], "cached": True, "key": key}
    space = candidates if candidates is not None else nat.furax_autotune_space()
    ms, best = nat.furax_autotune(P.handle, N.handle, _ACC[acc], space, reps)
    b = dict(space[best])
    b["kernel"] = _KERNELS[int(b["kernel"])]
    rec = {"schedule": b, "ms": ms[best], "candidates_timed": sum(1 for m in ms if m >= 0),
           "times_ms": [[_KERNELS[int(c["kernel"])], c["tile_len"], c["max_rows"], c["group_tol"],
                         int(c.get("l2_evict_first", 0)), int(c.get("consumer_warps", 0)), m]
                        for c, m in zip(space, ms)]}
    table[key] = rec
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1)
    os.replace(tmp, path)
    return {**rec, "cached": False, "key": key}

