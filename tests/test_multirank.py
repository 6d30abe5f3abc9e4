"""Host-side multi-rank logic of bench.py on two gloo ranks (CPU): the max-over-ranks timing,
the barrier, the whole-job value and the rank-0-only reference arm. Each rank of a multi-GPU
run solves its own replica of the workload, so no data-path collective exists to test."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 180.0][rank]                      # rank 1 is the slow one
    ms_max = bench.reduce_max(local_ms, world)
    bench.barrier(world)
    value = bench.job_value(1e9, 2, ms_max, world)
    q.put((rank, ms_max, value))
    dist.destroy_process_group()


def test_reduce_max_barrier_and_job_value():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms_max, value in got:
        assert ms_max == 180.0                           # every rank sees the slowest rank's time
        assert value == pytest.approx(2 * 1e9 * 2 / 0.180 / 1e9)


def test_job_value_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.job_value(268435456 * 50, 3, 1000.0, 1) == pytest.approx(268435456 * 50 * 3 / 1e9)


@pytest.mark.slow
def test_reference_arm_two_ranks_prints_once():
    """torchrun --nproc-per-node 2 bench.py --impl reference: rank 0 prints one JSON line, rank 1 nothing."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference", "--small",
           "--gpus", "2", "--steps", "1", "--warmup", "1"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["n_gpus"] == 2 and j["value"] > 0
    assert j["cpu_baseline"]["kind"] == "oracle" and j["e2e"]["h2d_bytes_per_step"] == 0
