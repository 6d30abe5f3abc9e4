"""GB300-native map-making hot path of linear-operator CMB analysis (Furax, arXiv 2603.19600).

The compute runs in libfurax.so (hand-written CUDA for sm_103a) behind a C ABI declared in
include/furax.h; this package binds it (``_native``, same names as the C entry points) and
adds a small object layer (``mapmaking``). There is no CPU fallback.
"""
from . import _native
from ._native import FuraxError, launch_count, version
from .mapmaking import (Chi2, Noise, Pointing, SolveInfo, Templates, autotune, blockdiag_precond, chi2, chi2_grad,
                        gapfill, mapmaker_cg, ptfp_apply, ptnp_apply, rhs)

__all__ = ["Pointing", "Noise", "SolveInfo", "Templates", "blockdiag_precond", "ptnp_apply", "ptfp_apply", "rhs",
           "mapmaker_cg", "chi2_grad", "gapfill", "autotune",
           "chi2", "Chi2", "FuraxError", "launch_count", "version", "_native"]
