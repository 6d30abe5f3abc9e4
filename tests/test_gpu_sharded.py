"""Detector sharding of a joint map: two processes (sharing the one GPU) each hold half of the
detectors and sum their partial P^T N^-1 P, right-hand side and preconditioner blocks through a
gloo all-reduce of host copies (the solver's allreduce callback). The sharded solve equals the
single-process solve over all detectors and the oracle's solve of the detector-concatenated
problem (the block decomposition P^T N^-1 P = sum_i P_i^T N_i^-1 P_i, "Algebraic reductions")."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch

import synth
from parity import rel

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("precision,mode,tol", [("f64", "cache_f64", 1e-9), ("f32", "cache_mixed", 1e-7)])
def test_sharded_solve_equals_joint_solve_and_oracle(fx, dev, orc, tmp_path, precision, mode, tol):
    nd, ns, nside = 12, 30000, 32
    o = synth.Observation(nside, synth.satellite_scan(ns, t0=900.0), synth.hex_focal_plane(nd))
    taps = np.tile(synth.inverse_noise_taps(), (nd, 1)) * np.linspace(0.8, 1.2, nd)[:, None]
    pix, c, s, _ = orc.pointing(nside, o.q_bore, o.q_det)
    g = synth.rng(95, 0)
    d = (orc.P(pix, c, s, synth.gaussian_sky(nside, g)) + synth.one_over_f_noise(nd, ns, g)).astype(np.float32)
    np.savez(tmp_path / "inputs.npz", q_bore=o.q_bore, q_det=o.q_det, taps=taps, d=d, nside=nside)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "tests", "sharded_worker.py"),
           str(tmp_path), precision, mode]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    x0, x1 = np.load(tmp_path / "x0.npy"), np.load(tmp_path / "x1.npy")
    v0, v1 = np.load(tmp_path / "v0.npy"), np.load(tmp_path / "v1.npy")
    i0 = json.load(open(tmp_path / "info0.json"))
    assert i0["converged"] and i0["allreduce_calls"] >= i0["iters"] + 3
    # every process ends with the same map (same sums, same vectors, same scalars)
    assert np.array_equal(x0, x1) and np.array_equal(v0, v1)
    # the single-process solve over all detectors
    P = fx.Pointing.from_observations([o], mode=mode, device=dev)
    N = fx.Noise.banded(P, taps)
    # both solved to 1e-12, as the oracle: the stopping point then does not decide the per-component
    # comparison (Q and U are ~100 times smaller than I)
    x, v, info = fx.mapmaker_cg(P, N, torch.as_tensor(d.ravel(), device=dev), maxiter=600, tol=1e-12,
                                precision=precision, acc="f32_kahan")
    assert info.converged
    v = v.cpu().numpy()
    assert np.array_equal(v, v0)
    assert rel(x0[v], x.cpu().numpy()[v], "sharded vs joint") < tol
    # the oracle's solve of the detector-concatenated problem
    on = orc.Noise(taps=taps)
    bj = orc.bj(o.npix, pix, c, s, on, 1e-3)
    assert np.array_equal(bj["valid"], v)
    b = orc.rhs(o.npix, pix, c, s, on, bj["valid"], d.astype(np.float64))
    xo, _, _ = orc.pcg(o.npix, pix, c, s, on, bj["valid"], bj["inv"], b, 400, 1e-12)
    assert rel(x0[v], xo[v], "sharded vs oracle") < tol
