"""The multi-GPU path of bench.py on CPU: replicas, no data-path collective.

With N ranks every rank solves the same workload; the bench line reports the DOF-iterations
of all ranks over the longest rank's time (sum and max over the process group).  Here two
`gloo` ranks on the CPU check that aggregation, and the reference arm's rule that only rank 0
runs the oracle under torchrun.
"""

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


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r processed 1000 (r + 1) DOF-iterations in 2 + r seconds
        units, secs = bench.aggregate(1000.0 * (rank + 1), 2.0 + rank, "cpu")
        out[rank] = (units, secs)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # every rank sees the sum of the units and the longest time
    assert out[0] == out[1] == (3000.0, 3.0)


def test_aggregate_without_a_process_group_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(123.0, 4.5) == (123.0, 4.5)


@pytest.mark.parametrize("rank", ["1", "3"])
def test_reference_arm_runs_on_rank_zero_only(rank):
    env = dict(os.environ, RANK=rank, LOCAL_RANK=rank, WORLD_SIZE="4")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "4"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
