"""FP64 CPU oracle for gap filling by constrained Gaussian realisation — TEST INFRASTRUCTURE.

The Furax paper ties its symmetric band Toeplitz operator to gap filling with constrained
Gaussian realisations (SymmetricBandToeplitzOperator, Table 2 and the text after it) without
stating the construction. This oracle takes the standard one: with N the noise covariance (a
symmetric band per detector), d the data, v the observed samples, g the gaps and n an
unconstrained realisation of covariance N (an input: the random draws of the method),

    d_g <- n_g + N_gv N_vv^-1 (d_v - n_v),    d_v unchanged,

i.e. the realisation conditioned on the observed samples. N_vv^-1 is applied by conjugate
gradients per detector with the pinned band product of this package. Only the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU leg may use it.

Parity status (pins in ``tests/test_oracle_gapfill.py``): pinned against the dense conditional
mean (numpy solve), and the special cases without gaps, with only gaps, with d = n and with a
white covariance (no correlation to borrow from).
"""
from __future__ import annotations

import numpy as np

from . import ninv_band


def gapfill(cov_taps, d, valid, n, maxiter=1000, tol=1e-12):
    """Fill the gaps (valid == False) of d [ndet][ns] with the constrained realisation; returns
    (filled TOD, PCG iterations per detector). cov_taps [ndet][K] is the covariance band."""
    cov_taps = np.atleast_2d(np.asarray(cov_taps, np.float64))
    d = np.asarray(d, np.float64)
    n = np.asarray(n, np.float64)
    valid = np.asarray(valid, bool)
    out = d.copy()
    iters = []
    for i in range(d.shape[0]):
        v = valid[i]
        band = cov_taps[i:i + 1]

        def nvv(y):
            return np.where(v, ninv_band(band, np.where(v, y, 0.0)[None, :])[0], 0.0)

        r = np.where(v, d[i] - n[i], 0.0)
        y = np.zeros_like(r)
        p = r.copy()
        rr = float(r @ r)
        rr0 = rr
        it = 0
        while it < maxiter and rr > tol * tol * rr0:
            q = nvv(p)
            alpha = rr / float(p @ q)
            y += alpha * p
            r -= alpha * q
            rr_new = float(r @ r)
            p = r + (rr_new / rr) * p
            rr = rr_new
            it += 1
        fill = n[i] + ninv_band(band, y[None, :])[0]
        out[i] = np.where(v, d[i], fill)
        iters.append(it)
    return out, np.array(iters)
