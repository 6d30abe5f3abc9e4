"""FP64 CPU oracle for template deprojection — TEST INFRASTRUCTURE.

Plain numpy restatement of the weighting-and-deprojection operator of the Furax paper
(Statement of Need: the generalised least-squares estimator
m = (H^T F_T H)^-1 H^T F_T d with F_T = W - W T (T^T W T)^-1 T^T W, and the
TemplateOperator of Table 3), built on the pinned primitives of this package (P, P^T, N^-1).
Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU leg may use it; it shares
nothing with the CUDA library.

Conventions the paper leaves open (it names templates but does not fix them):
  * T, per detector: the Legendre polynomials P_0 .. P_K (K = ``order`` <= 3) of the scaled
    time tau_t = 2 t / (ns - 1) - 1 over that detector's whole stream (tau = 0 when ns = 1);
  * W is the inverse noise covariance N^-1 of the noise model (white or the symmetric band);
  * F_T acts on each detector's stream separately (T and W are block-diagonal in detectors).

Parity status (pins in ``tests/test_oracle_templates.py``):
  legendre_templates      pinned (numpy.polynomial.legendre, closed forms P_1..P_3)
  gram / deproject        pinned (white noise: residual of numpy.polyfit; F_T T = 0; symmetry;
                          dense matrices; F_T W^-1 F_T = F_T)
  ptfp_apply / rhs / pcg  pinned (dense normal equations, invariance under d -> d + T alpha,
                          white noise + offsets = mean-subtracted binned solve)
"""
from __future__ import annotations

import numpy as np

from . import P, PT, Noise, bj_apply

MAX_ORDER = 3


def legendre_templates(ns: int, order: int) -> np.ndarray:
    """T [ns][order+1]: P_0..P_order at tau_t = 2t/(ns-1) - 1, by the three-term recurrence
    (n+1) P_{n+1} = (2n+1) tau P_n - n P_{n-1}."""
    assert 0 <= order <= MAX_ORDER and ns >= 1
    tau = np.zeros(ns) if ns == 1 else 2.0 * np.arange(ns) / (ns - 1) - 1.0
    T = np.empty((ns, order + 1))
    T[:, 0] = 1.0
    if order >= 1:
        T[:, 1] = tau
    for n in range(1, order):
        T[:, n + 1] = ((2 * n + 1) * tau * T[:, n] - n * T[:, n - 1]) / (n + 1)
    return T


def weighted_templates(noise: Noise, ndet: int, ns: int, order: int) -> np.ndarray:
    """W T per detector [ndet][order+1][ns]: N^-1 applied to each template column."""
    T = legendre_templates(ns, order)
    cols = [noise.apply(np.tile(T[:, l], (ndet, 1))) for l in range(order + 1)]
    return np.stack(cols, axis=1)


def gram(noise: Noise, ndet: int, ns: int, order: int) -> np.ndarray:
    """G [ndet][order+1][order+1] = T^T W T per detector."""
    T = legendre_templates(ns, order)
    WT = weighted_templates(noise, ndet, ns, order)
    return np.einsum("tk,dlt->dkl", T, WT)


def deproject(noise: Noise, order: int, x: np.ndarray) -> np.ndarray:
    """y = F_T x = W x - W T (T^T W T)^-1 T^T W x for a TOD x [ndet][ns], detector by detector."""
    x = np.asarray(x, np.float64)
    ndet, ns = x.shape
    T = legendre_templates(ns, order)
    z = noise.apply(x)                       # W x
    a = z @ T                                # T^T W x            [ndet][K+1]
    G = gram(noise, ndet, ns, order)
    b = np.stack([np.linalg.solve(G[i], a[i]) for i in range(ndet)])
    WT = weighted_templates(noise, ndet, ns, order)
    return z - np.einsum("dlt,dl->dt", WT, b)


def _mask(valid, m):
    return m if valid is None else np.where(np.asarray(valid, bool)[:, None], m, 0.0)


def ptfp_apply(npix, pix, c, s, noise: Noise, order: int, valid, x):
    """S P^T F_T P S^T x (S: the valid-pixel mask, None = all pixels)."""
    tod = P(pix, c, s, _mask(valid, np.asarray(x, np.float64)))
    y = deproject(noise, order, tod)
    return _mask(valid, PT(npix, pix, c, s, y)[0])


def rhs(npix, pix, c, s, noise: Noise, order: int, valid, d):
    """S P^T F_T d."""
    y = deproject(noise, order, np.asarray(d, np.float64))
    return _mask(valid, PT(npix, pix, c, s, y)[0])


def pcg(npix, pix, c, s, noise: Noise, order: int, valid, minv, b, maxiter, tol=1e-8):
    """Preconditioned CG for S P^T F_T P S^T x = b from x = 0 with the block preconditioner
    minv (the 3x3 inverses of ``oracle.bj``). Stops when ||r|| <= tol ||b||. Returns
    (x, iterations, residual history)."""
    v = np.asarray(valid, bool)

    def prec(r):
        return bj_apply(minv, v, r)

    def A(p):
        return ptfp_apply(npix, pix, c, s, noise, order, v, p)

    b = _mask(v, np.asarray(b, np.float64))
    x = np.zeros((npix, 3))
    r = b.copy()
    z = prec(r)
    p = z.copy()
    rz = float(np.sum(r * z))
    bb = float(np.sum(b * b))
    hist = [np.sqrt(float(np.sum(r * r)) / bb) if bb > 0 else 0.0]
    it = 0
    while it < maxiter and hist[-1] > tol:
        q = A(p)
        alpha = rz / float(np.sum(p * q))
        x += alpha * p
        r -= alpha * q
        it += 1
        hist.append(np.sqrt(float(np.sum(r * r)) / bb))
        if hist[-1] <= tol:
            break
        z = prec(r)
        rz_new = float(np.sum(r * z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, np.array(hist)
