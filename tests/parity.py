"""Element-wise comparison of GPU results with the FP64 oracle (test infrastructure).

Two measures, both per element rather than through a global L2 norm:

* ``rel(got, ref)``: for a map ``[npix][3]`` the largest absolute error of each Stokes
  component divided by that component's largest reference magnitude, maximised over the
  components; for any other array the largest absolute error over the largest reference
  magnitude. One pixel that is off shows up at its own size, whatever the map's size.
* ``elem(got, ref, scale)``: ``max_i |got_i - ref_i| / scale_i`` with ``scale`` the same
  operation applied to absolute values (``|A| |x|``), the quantity that the standard
  floating-point error bound ``|fl(A x) - A x| <= gamma_k |A| |x|`` is stated against.

Both also compute the L2 error per component; with ``FURAX_PARITY_LOG`` set to a file name
every comparison appends one JSON line (test id, label, measures, tolerance if given), so a
run records the margin of every bound.
"""
from __future__ import annotations

import json
import os

import numpy as np


def _np(a):
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.asarray(a, dtype=np.float64)


def _is_map(a: np.ndarray) -> bool:
    return a.ndim == 2 and a.shape[1] == 3


def _log(kind: str, out: dict, label: str | None):
    path = os.environ.get("FURAX_PARITY_LOG")
    if not path:
        return
    rec = {"test": os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0], "kind": kind, "label": label, **out}
    with open(path, "a") as f:
        f.write(json.dumps(rec) + "\n")


def errors(got, ref) -> dict:
    """Per-component max-abs error, scale (max |ref|) and L2 relative error."""
    g, r = _np(got), _np(ref)
    if g.shape != r.shape:
        raise AssertionError(f"shape {g.shape} != {r.shape}")
    cols = [(g[:, k], r[:, k]) for k in range(3)] if _is_map(r) else [(g.ravel(), r.ravel())]
    out = {"max_abs": [], "scale": [], "max_rel": [], "l2_rel": []}
    for gc, rc in cols:
        d = np.abs(gc - rc)
        mx = float(d.max()) if d.size else 0.0
        sc = float(np.abs(rc).max()) if rc.size else 0.0
        l2 = float(np.linalg.norm(gc - rc) / max(np.linalg.norm(rc), 1e-300))
        out["max_abs"].append(mx)
        out["scale"].append(sc)
        out["max_rel"].append(mx / sc if sc > 0 else (0.0 if mx == 0 else np.inf))
        out["l2_rel"].append(l2)
    return out


def rel(got, ref, label: str | None = None) -> float:
    """Largest per-component (max-abs error / max |reference|)."""
    e = errors(got, ref)
    _log("rel", e, label)
    return max(e["max_rel"]) if e["max_rel"] else 0.0


def elem(got, ref, scale, label: str | None = None, floor: float = 0.0) -> float:
    """max_i |got_i - ref_i| / scale_i; elements with scale_i <= floor must match to within floor."""
    g, r, s = _np(got).ravel(), _np(ref).ravel(), _np(scale).ravel()
    d = np.abs(g - r)
    big = s > floor
    worst = float((d[big] / s[big]).max()) if big.any() else 0.0
    small = float(d[~big].max()) if (~big).any() else 0.0
    out = {"max_scaled": worst, "max_abs_where_scale_small": small, **errors(got, ref)}
    _log("elem", out, label)
    if small > floor:
        return np.inf
    return worst
