"""One process of the detector-sharding test (test_gpu_sharded.py), launched by torchrun.

Every process solves the same map from its own subset of the detectors (detector d goes to process
d mod world): the solver sums the preconditioner blocks and hits, the right-hand side and every
application of the normal operator over the processes through the allreduce callback, here a gloo
all-reduce of host copies. Inputs come from the test's directory; the map is written back there."""
import json
import os
import sys

import numpy as np
import torch
import torch.distributed as dist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    work, precision, mode = sys.argv[1], sys.argv[2], sys.argv[3]
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo")
    torch.cuda.set_device(0)
    import paper_2603_19600_gb300 as fx
    inp = np.load(os.path.join(work, "inputs.npz"))
    nside = int(inp["nside"])
    dets = np.arange(rank, inp["q_det"].shape[0], world)
    dev = torch.device("cuda", 0)
    P = fx.Pointing(torch.as_tensor(inp["q_bore"], device=dev), torch.as_tensor(inp["q_det"][dets], device=dev),
                    [len(dets)], [inp["q_bore"].shape[0]], [nside], mode=mode)
    N = fx.Noise.banded(P, inp["taps"][dets])
    d = torch.as_tensor(np.ascontiguousarray(inp["d"][dets]).ravel(), device=dev)
    calls = []

    def allreduce(t):
        calls.append(int(t.numel()))
        host = t.cpu()
        dist.all_reduce(host)
        t.copy_(host)

    x, v, info = fx.mapmaker_cg(P, N, d, maxiter=600, tol=1e-12, precision=precision, acc="f32_kahan",
                                allreduce=allreduce)
    np.save(os.path.join(work, f"x{rank}.npy"), x.cpu().numpy())
    np.save(os.path.join(work, f"v{rank}.npy"), v.cpu().numpy())
    with open(os.path.join(work, f"info{rank}.json"), "w") as f:
        json.dump({"iters": info.iters, "converged": info.converged, "true_rel_res": info.true_rel_res,
                   "allreduce_calls": len(calls), "dets": dets.tolist()}, f)
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
