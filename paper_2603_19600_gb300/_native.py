"""ctypes binding of libfurax.so: one Python function per C entry point, same names.

Arguments are torch tensors on the current CUDA device (or plain Python values); each
function checks dtype, device, contiguity and size, passes ``tensor.data_ptr()`` and
``torch.cuda.current_stream().cuda_stream``, and raises FuraxError on a negative status.
There is no fallback: if the library is not built, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

FURAX_OK = 0
FURAX_ENOTCONVERGED = 1
FURAX_F32, FURAX_F64 = 0, 1
FURAX_ACC_F64, FURAX_ACC_F32_KAHAN, FURAX_ACC_F32 = 0, 1, 2
FURAX_POINTING_ON_THE_FLY, FURAX_POINTING_CACHE_F32, FURAX_POINTING_CACHE_F64, FURAX_POINTING_CACHE_MIXED = 0, 1, 2, 3
FURAX_PREC_F32X2 = 2
FURAX_NOISE_WHITE, FURAX_NOISE_BANDED = 0, 1

_DT = {torch.float32: FURAX_F32, torch.float64: FURAX_F64}


class FuraxError(RuntimeError):
    def __init__(self, func: str, code: int, msg: str):
        super().__init__(f"{func} failed with status {code}: {msg}")
        self.code = code


class ObsDesc(ctypes.Structure):
    _fields_ = [("n_obs", ctypes.c_int32), ("ndet", ctypes.c_void_p), ("nsamp", ctypes.c_void_p),
                ("nside", ctypes.c_void_p), ("q_bore", ctypes.c_void_p), ("q_det", ctypes.c_void_p),
                ("psi_offset", ctypes.c_void_p), ("hwp_angle", ctypes.c_void_p), ("map_id", ctypes.c_void_p)]


class CgOpts(ctypes.Structure):
    _fields_ = [("maxiter", ctypes.c_int32), ("tol", ctypes.c_double), ("precision", ctypes.c_int32),
                ("acc", ctypes.c_int32), ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("check_every", ctypes.c_int32), ("rcond_min", ctypes.c_double),
                ("binned_only", ctypes.c_int32), ("true_residual", ctypes.c_int32), ("d_ready", ctypes.c_void_p),
                ("allreduce", ctypes.c_void_p), ("allreduce_user", ctypes.c_void_p)]


FURAX_REDUCE_F64, FURAX_REDUCE_I32 = 0, 1
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                ctypes.c_void_p)


class _DeviceView:
    """A device buffer of the library exposed through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr: int, n: int, dtype: int):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8" if dtype == FURAX_REDUCE_F64 else "<i4",
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def allreduce_callback(fn):
    """Wrap fn(tensor) -> None, which sums a CUDA tensor in place over the processes of a sharded map
    (on the current stream), as a furax_allreduce_fn. Keep the returned object alive during the solve."""

    def cb(buf, n, dtype, stream, user):
        try:
            fn(torch.as_tensor(_DeviceView(buf, n, dtype), device=torch.device("cuda", torch.cuda.current_device())))
            return 0
        except Exception:  # noqa: BLE001 - reported to the solver as a status, which raises
            return -3

    return ALLREDUCE_FN(cb)


class Schedule(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("tile_len", ctypes.c_int32), ("max_rows", ctypes.c_int32),
                ("group_tol", ctypes.c_double), ("l2_evict_first", ctypes.c_int32), ("consumer_warps", ctypes.c_int32)]


FURAX_SCHED_TIME_ORDERED, FURAX_SCHED_PIXEL_SORTED = 0, 1


class CgResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("outer", ctypes.c_int32), ("rel_res", ctypes.c_double),
                ("true_rel_res", ctypes.c_double), ("n_valid", ctypes.c_int64),
                ("hist", ctypes.POINTER(ctypes.c_double)), ("hist_len", ctypes.c_int32),
                ("hist_written", ctypes.c_int32)]


_V, _I32, _I64, _D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_SIGS = {
    "furax_pointing_create": [ctypes.POINTER(ObsDesc), _I32, _V, ctypes.POINTER(_V)],
    "furax_pointing_destroy": [_V],
    "furax_pointing_info": [_V, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
    "furax_pointing_refresh": [_V, _V],
    "furax_pointing_cache": [_V, _V, _V, _V, _V],
    "furax_device_status": [_V, _V],
    "furax_set_wait_budget": [_V, _I64, _V],
    "furax_pointing_set_schedule": [_V, ctypes.POINTER(Schedule), _V],
    "furax_pointing_get_schedule": [_V, ctypes.POINTER(Schedule)],
    "furax_autotune": [_V, _V, _I32, ctypes.POINTER(Schedule), _I32, _I32, ctypes.POINTER(_D),
                       ctypes.POINTER(_I32), _V],
    "furax_autotune_space": [ctypes.POINTER(Schedule), _I32],
    "furax_probe_convert": [_V, _V, _V, _V, _I64, _V],
    "furax_probe_fma": [_I32, _I64, _V, ctypes.POINTER(_D), _V],
    "furax_probe_l2": [_I32, _V, _I64, _V, _I64, _V, _V],
    "furax_debug_hold_loader": [_V, _I32, _V],
    "furax_pointing_set_psi_offset": [_V, _V, _V],
    "furax_profile_read": [_I32, ctypes.POINTER(_D), ctypes.POINTER(_I64)],
    "furax_pointing_expand": [_V, _V, _V, _V, _I32, _V],
    "furax_pointing_apply": [_V, _V, _I32, _V, _I32, _V],
    "furax_pointing_transpose": [_V, _V, _I32, _V, _I32, _I32, _V, _I32, _V],
    "furax_noise_create": [_I32, _V, _I32, ctypes.POINTER(ObsDesc), _V, ctypes.POINTER(_V)],
    "furax_noise_destroy": [_V],
    "furax_noise_inv_apply": [_V, _V, _V, _I32, _V],
    "furax_blockdiag_precond": [_V, _V, _D, _V, _V, _V, _V, _V],
    "furax_ptnp_apply": [_V, _V, _V, _V, _V, _I32, _I32, _V],
    "furax_rhs": [_V, _V, _V, _I32, _V, _V, _V],
    "furax_ptnp_apply_noalloc": [_V, _V, _V, _I32, _I64, _I32, _V, _I32, _V, _V, _V, _V],
    "furax_mapmaker_cg": [_V, _V, _V, _I32, _V, _V, ctypes.POINTER(CgOpts), ctypes.POINTER(CgResult), _V],
    "furax_chi2_grad": [_V, _V, _V, _I32, _V, _V, _V, _V, _I32, _V],
    "furax_gapfill": [_V, _V, _V, _V, _V, _I32, _I32, _D, _I32, _V, _V],
    "furax_templates_create": [_V, _V, _I32, _V, ctypes.POINTER(_V)],
    "furax_templates_destroy": [_V],
    "furax_templates_gram": [_V, _V, _V],
    "furax_deproject_apply": [_V, _V, _V, _I32, _V],
    "furax_ptfp_apply": [_V, _V, _V, _V, _I32, _I32, _V],
    "furax_mapmaker_cg_deproject": [_V, _V, _I32, _V, _V, ctypes.POINTER(CgOpts), ctypes.POINTER(CgResult), _V, _V],
}

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB_PATH


def lib() -> ctypes.CDLL:
    """Load libfurax.so. Raises if it has not been built: there is no CPU path."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libfurax.so not found at {path}: build it with "
                                   "paper_2603_19600_gb300.build.build() (needs nvcc)")
            torch.cuda.init()
            l = ctypes.CDLL(path)
            for name, args in _SIGS.items():
                f = getattr(l, name)
                f.argtypes = args
                f.restype = ctypes.c_int32
            l.furax_last_error.restype = ctypes.c_char_p
            l.furax_launch_count.restype = ctypes.c_int64
            l.furax_version.restype = ctypes.c_char_p
            l.furax_cg_default_opts.argtypes = [ctypes.POINTER(CgOpts)]
            l.furax_cg_default_opts.restype = None
            l.furax_profile_enable.argtypes = [ctypes.c_int32]
            l.furax_profile_enable.restype = None
            l.furax_profile_reset.restype = None
            _lib = l
    return _lib


def _call(name: str, *args, ok=(FURAX_OK,)) -> int:
    rc = getattr(lib(), name)(*args)
    if rc < 0 or (rc not in ok and rc < 0):
        raise FuraxError(name, rc, lib().furax_last_error().decode())
    return rc


def _stream(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _ptr(t: torch.Tensor | None, dtype=None, numel=None, name="tensor") -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t.data_ptr()


def _dt(t: torch.Tensor) -> int:
    if t.dtype not in _DT:
        raise ValueError(f"unsupported dtype {t.dtype}")
    return _DT[t.dtype]


def launch_count() -> int:
    return int(lib().furax_launch_count())


def version() -> str:
    return lib().furax_version().decode()


def default_cg_opts() -> CgOpts:
    o = CgOpts()
    lib().furax_cg_default_opts(ctypes.byref(o))
    return o


class _Desc:
    """Keeps the host arrays of an ObsDesc alive."""

    def __init__(self, ndet, nsamp, nside, q_bore=None, q_det=None, psi_offset=None, hwp_angle=None, map_id=None):
        self.n = len(ndet)
        self.ndet = (ctypes.c_int32 * self.n)(*[int(v) for v in ndet])
        self.nsamp = (ctypes.c_int64 * self.n)(*[int(v) for v in nsamp])
        self.nside = (ctypes.c_int32 * self.n)(*[int(v) for v in nside])
        self.map_id = None if map_id is None else (ctypes.c_int32 * self.n)(*[int(v) for v in map_id])
        self.desc = ObsDesc(self.n, ctypes.cast(self.ndet, _V), ctypes.cast(self.nsamp, _V),
                            ctypes.cast(self.nside, _V), q_bore, q_det, psi_offset, hwp_angle,
                            None if self.map_id is None else ctypes.cast(self.map_id, _V))


# ------------------------------------------------------------------ entry points, same names as the C ABI
def furax_pointing_create(q_bore, q_det, ndet, nsamp, nside, psi_offset=None, mode=FURAX_POINTING_CACHE_F32,
                          stream=None, hwp_angle=None, map_id=None) -> int:
    nb, nd = sum(int(v) for v in nsamp), sum(int(v) for v in ndet)
    if map_id is not None and len(map_id) != len(ndet):
        raise ValueError("map_id needs one entry per observation")
    d = _Desc(ndet, nsamp, nside, _ptr(q_bore, torch.float64, 4 * nb, "q_bore"),
              _ptr(q_det, torch.float64, 4 * nd, "q_det"), _ptr(psi_offset, torch.float64, nd, "psi_offset"),
              _ptr(hwp_angle, torch.float64, nb, "hwp_angle"), map_id)
    h = _V()
    _call("furax_pointing_create", ctypes.byref(d.desc), mode, _stream(stream), ctypes.byref(h))
    return h.value


def furax_pointing_destroy(h) -> None:
    if h:
        _call("furax_pointing_destroy", h)


def furax_pointing_info(h):
    a, b, c, d = _I64(), _I64(), _I64(), _I64()
    _call("furax_pointing_info", h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d))
    return dict(nsamp_total=a.value, npix_total=b.value, ndet_total=c.value, n_invalid=d.value)


def furax_pointing_refresh(h, stream=None) -> None:
    _call("furax_pointing_refresh", h, _stream(stream))


def furax_device_status(h, stream=None) -> None:
    """Raise FuraxError (FURAX_ETIMEOUT) if a bounded device-side wait gave up."""
    _call("furax_device_status", h, _stream(stream))


def furax_pointing_set_schedule(h, kernel: int, tile_len: int = 0, max_rows: int = 12, group_tol: float = 2.0,
                                l2_evict_first: int = 0, consumer_warps: int = 0, stream=None) -> None:
    sch = Schedule(int(kernel), int(tile_len), int(max_rows), float(group_tol), int(l2_evict_first),
                   int(consumer_warps))
    _call("furax_pointing_set_schedule", h, ctypes.byref(sch), _stream(stream))


def furax_pointing_get_schedule(h) -> dict:
    sch = Schedule()
    _call("furax_pointing_get_schedule", h, ctypes.byref(sch))
    return dict(kernel=sch.kernel, tile_len=sch.tile_len, max_rows=sch.max_rows, group_tol=sch.group_tol,
                l2_evict_first=sch.l2_evict_first, consumer_warps=sch.consumer_warps)


def furax_autotune_space() -> list:
    n = lib().furax_autotune_space(None, 0)
    arr = (Schedule * n)()
    lib().furax_autotune_space(arr, n)
    return [dict(kernel=c.kernel, tile_len=c.tile_len, max_rows=c.max_rows, group_tol=c.group_tol,
                 l2_evict_first=c.l2_evict_first, consumer_warps=c.consumer_warps) for c in arr]


def furax_autotune(hp, hn, acc: int, candidates: list, reps: int = 3, stream=None):
    """Time each candidate schedule (dicts of furax_schedule fields); returns (ms per candidate, best index)."""
    n = len(candidates)
    arr = (Schedule * n)(*[Schedule(int(c["kernel"]), int(c["tile_len"]), int(c["max_rows"]), float(c["group_tol"]),
                                    int(c.get("l2_evict_first", 0)), int(c.get("consumer_warps", 0)))
                           for c in candidates])
    ms = (ctypes.c_double * n)()
    best = _I32()
    _call("furax_autotune", hp, hn, int(acc), arr, n, int(reps), ms, ctypes.byref(best), _stream(stream))
    return [ms[i] for i in range(n)], best.value


def furax_set_wait_budget(h, cycles: int, stream=None) -> None:
    """Budget (SM cycles) of the handle's bounded device waits; 0 restores the default."""
    _call("furax_set_wait_budget", h, int(cycles), _stream(stream))


def furax_debug_hold_loader(h, hold: bool, stream=None) -> None:
    """Test hook: hold the cached FP32 operator's loader so that its other roles' waits run out."""
    _call("furax_debug_hold_loader", h, int(bool(hold)), _stream(stream))


def furax_probe_convert(in64=None, out32=None, in32=None, out64=None, stream=None) -> None:
    """Encoding-level conversions: out32 = binary32(in64) (nearest even), out64 = binary64(in32)."""
    n = (in64 if in64 is not None else in32).numel()
    _call("furax_probe_convert", _ptr(in64, torch.float64, n, "in64"), _ptr(out32, torch.float32, n, "out32"),
          _ptr(in32, torch.float32, n, "in32"), _ptr(out64, torch.float64, n, "out64"), n, _stream(stream))


def furax_probe_fma(kind: int, iters: int, sink, stream=None) -> float:
    """Launch the FMA throughput probe (0 FP64, 1 FP32, 2 packed FP32); returns its flop count."""
    fl = _D()
    _call("furax_probe_fma", int(kind), int(iters), _ptr(sink, None, None, "sink"), ctypes.byref(fl), _stream(stream))
    return fl.value


def furax_probe_l2(kind: int, idx, table, ntable: int, sink, stream=None) -> None:
    """Random L2 operations at idx (int32, each in [0, ntable)) on table (see furax.h for its size)."""
    if idx.numel() and (int(idx.min()) < 0 or int(idx.max()) >= ntable):
        raise ValueError("probe indices must lie in [0, ntable)")
    need = {0: 16 * ntable, 1: 16 * ntable, 2: 32 * ntable, 3: 24 * ntable, 4: 32 * ntable, 5: 24 * ntable,
            6: 24 * ntable, 7: 16 * ntable, 8: 24 * ntable}[int(kind)]
    if table.numel() * table.element_size() < need:
        raise ValueError(f"probe table needs {need} bytes")
    _call("furax_probe_l2", int(kind), _ptr(idx, torch.int32, None, "idx"), idx.numel(), _ptr(table, None, None, "table"),
          int(ntable), _ptr(sink, None, None, "sink"), _stream(stream))


def furax_profile_enable(on: bool) -> None:
    lib().furax_profile_enable(int(bool(on)))


def furax_profile_reset() -> None:
    lib().furax_profile_reset()


def furax_profile_read(kernel: int):
    """(total milliseconds, number of timed launches) of kernel 0 (FP32 fused) or 1 (FP64 fused)."""
    ms, n = _D(), _I64()
    _call("furax_profile_read", kernel, ctypes.byref(ms), ctypes.byref(n))
    return ms.value, n.value


def furax_pointing_set_psi_offset(h, psi_offset, stream=None) -> None:
    _call("furax_pointing_set_psi_offset", h, _ptr(psi_offset, torch.float64, None, "psi_offset"), _stream(stream))


def furax_pointing_expand(h, pix, c, s, stream=None) -> None:
    _call("furax_pointing_expand", h, _ptr(pix, torch.int32, None, "pix"), _ptr(c, None, pix.numel(), "c"),
          _ptr(s, c.dtype, pix.numel(), "s"), _dt(c), _stream(stream))


def furax_pointing_cache(h, pix, c, s, stream=None) -> None:
    _call("furax_pointing_cache", h, _ptr(pix, torch.int32, None, "pix"), _ptr(c, torch.float32, pix.numel(), "c"),
          _ptr(s, torch.float32, pix.numel(), "s"), _stream(stream))


def furax_pointing_apply(h, m, tod, stream=None) -> None:
    _call("furax_pointing_apply", h, _ptr(m, None, None, "map"), _dt(m), _ptr(tod, None, None, "tod"), _dt(tod),
          _stream(stream))


def furax_pointing_transpose(h, tod, m, acc=FURAX_ACC_F64, hits=None, accumulate=False, stream=None) -> None:
    _call("furax_pointing_transpose", h, _ptr(tod, None, None, "tod"), _dt(tod), _ptr(m, None, None, "map"), _dt(m),
          acc, _ptr(hits, torch.int32, None, "hits"), int(bool(accumulate)), _stream(stream))


def furax_noise_create(kind, params, ntaps, ndet, nsamp, nside, stream=None) -> int:
    d = _Desc(ndet, nsamp, nside)
    h = _V()
    _call("furax_noise_create", kind, _ptr(params, torch.float64, None, "params"), ntaps, ctypes.byref(d.desc),
          _stream(stream), ctypes.byref(h))
    return h.value


def furax_noise_destroy(h) -> None:
    if h:
        _call("furax_noise_destroy", h)


def furax_noise_inv_apply(h, x, out, stream=None) -> None:
    if x.dtype != out.dtype:
        raise ValueError("in and out must have the same dtype")
    _call("furax_noise_inv_apply", h, _ptr(x, None, None, "in"), _ptr(out, None, x.numel(), "out"), _dt(x),
          _stream(stream))


def furax_blockdiag_precond(hp, hn, rcond_min, blocks_inv, valid, hits=None, rcond=None, stream=None) -> None:
    _call("furax_blockdiag_precond", hp, hn, float(rcond_min), _ptr(blocks_inv, torch.float64, None, "blocks_inv"),
          _ptr(valid, torch.uint8, None, "valid"), _ptr(hits, torch.int32, None, "hits"),
          _ptr(rcond, torch.float64, None, "rcond"), _stream(stream))


def furax_ptnp_apply(hp, hn, x, out, valid=None, precision=FURAX_F32, acc=FURAX_ACC_F32, stream=None) -> None:
    _call("furax_ptnp_apply", hp, hn, _ptr(x, torch.float64, None, "x"), _ptr(out, torch.float64, x.numel(), "out"),
          _ptr(valid, torch.uint8, None, "valid"), precision, acc, _stream(stream))


def furax_ptnp_apply_noalloc(pix, c, s, ndet, nsamp, nside, taps, x, out, valid=None, stream=None) -> None:
    """out = S P^T N^-1 P S^T x in FP32 for callers that cannot allocate (see include/furax.h)."""
    n = int(ndet) * int(nsamp)
    _call("furax_ptnp_apply_noalloc", _ptr(pix, torch.int32, n, "pix"), _ptr(c, torch.float32, n, "c"),
          _ptr(s, torch.float32, n, "s"), int(ndet), int(nsamp), int(nside), _ptr(taps, torch.float32, None, "taps"),
          taps.numel() // int(ndet), _ptr(valid, torch.uint8, None, "valid"), _ptr(x, torch.float64, None, "x"),
          _ptr(out, torch.float64, x.numel(), "out"), _stream(stream))


def furax_rhs(hp, hn, d, b, valid=None, stream=None) -> None:
    _call("furax_rhs", hp, hn, _ptr(d, None, None, "d"), _dt(d), _ptr(valid, torch.uint8, None, "valid"),
          _ptr(b, torch.float64, None, "b"), _stream(stream))


def furax_mapmaker_cg(hp, hn, d, x, valid=None, opts: CgOpts | None = None, hist_len=0, stream=None):
    o = opts if opts is not None else default_cg_opts()
    res = CgResult()
    hist = (ctypes.c_double * max(hist_len, 1))()
    res.hist = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double)) if hist_len > 0 else None
    res.hist_len = hist_len
    rc = _call("furax_mapmaker_cg", hp, hn, _ptr(d, None, None, "d"), _dt(d), _ptr(x, torch.float64, None, "x"),
               _ptr(valid, torch.uint8, None, "valid"), ctypes.byref(o), ctypes.byref(res), _stream(stream),
               ok=(FURAX_OK, FURAX_ENOTCONVERGED))
    return rc, res, [hist[i] for i in range(res.hist_written)]


def furax_gapfill(hn, ndet, d, valid, n_real, out, maxiter=1000, tol=1e-10, precision=FURAX_F64, stream=None):
    """Returns (status, per-detector iterations); ndet = detectors of the handle."""
    if not (d.dtype == n_real.dtype == out.dtype):
        raise ValueError("d, n_real and out must have one dtype")
    iters = (ctypes.c_int32 * max(int(ndet), 1))()
    rc = _call("furax_gapfill", hn, _ptr(d, None, None, "d"), _ptr(valid, torch.uint8, d.numel(), "valid"),
               _ptr(n_real, None, d.numel(), "n_real"), _ptr(out, None, d.numel(), "out"), _dt(d), int(maxiter),
               float(tol), int(precision), iters, _stream(stream), ok=(FURAX_OK, FURAX_ENOTCONVERGED))
    return rc, [iters[i] for i in range(ndet)]


def furax_templates_create(hp, hn, order, stream=None) -> int:
    h = _V()
    _call("furax_templates_create", hp, hn, int(order), _stream(stream), ctypes.byref(h))
    return h.value


def furax_templates_destroy(h) -> None:
    if h:
        _call("furax_templates_destroy", h)


def furax_templates_gram(h, gram, stream=None) -> None:
    _call("furax_templates_gram", h, _ptr(gram, torch.float64, None, "gram"), _stream(stream))


def furax_deproject_apply(h, x, out, stream=None) -> None:
    if x.dtype != out.dtype:
        raise ValueError("in and out must have the same dtype")
    _call("furax_deproject_apply", h, _ptr(x, None, None, "in"), _ptr(out, None, x.numel(), "out"), _dt(x),
          _stream(stream))


def furax_ptfp_apply(ht, x, out, valid=None, precision=FURAX_F32, acc=FURAX_ACC_F32, stream=None) -> None:
    _call("furax_ptfp_apply", ht, _ptr(x, torch.float64, None, "x"), _ptr(out, torch.float64, x.numel(), "out"),
          _ptr(valid, torch.uint8, None, "valid"), precision, acc, _stream(stream))


def furax_mapmaker_cg_deproject(ht, d, x, valid=None, opts: CgOpts | None = None, hist_len=0, amplitudes=None,
                                stream=None):
    o = opts if opts is not None else default_cg_opts()
    res = CgResult()
    hist = (ctypes.c_double * max(hist_len, 1))()
    res.hist = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double)) if hist_len > 0 else None
    res.hist_len = hist_len
    rc = _call("furax_mapmaker_cg_deproject", ht, _ptr(d, None, None, "d"), _dt(d), _ptr(x, torch.float64, None, "x"),
               _ptr(valid, torch.uint8, None, "valid"), ctypes.byref(o), ctypes.byref(res),
               _ptr(amplitudes, torch.float64, None, "amplitudes"), _stream(stream), ok=(FURAX_OK, FURAX_ENOTCONVERGED))
    return rc, res, [hist[i] for i in range(res.hist_written)]


def furax_chi2_grad(hp, hn, d, m, chi2, grad_map=None, grad_psi=None, precision=FURAX_F64, stream=None) -> None:
    _call("furax_chi2_grad", hp, hn, _ptr(d, None, None, "d"), _dt(d), _ptr(m, torch.float64, None, "m"),
          _ptr(chi2, torch.float64, None, "chi2"), _ptr(grad_map, torch.float64, None, "grad_map"),
          _ptr(grad_psi, torch.float64, None, "grad_psi"), precision, _stream(stream))
