"""The multi-process replica path of bench.py on the CPU (gloo, world size 2):
each rank runs an independent replica, the job time is the slowest rank's and
the throughput counts the units of all ranks.  No GPU is involved."""

import os
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took 10 (r + 1) ms for 5 steps of 1000 units each
    ms_step, value = bench.replica_throughput(10.0 * (rank + 1), 1000, 5, world, "cpu")
    e2e = bench.replica_max_ms(3.0 + rank, world, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, f"r{rank}.txt"), "w") as f:
        f.write(f"{ms_step} {value} {e2e}")


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_units(tmp_path):
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    for r in range(2):
        ms_step, value, e2e = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert ms_step == pytest.approx(4.0)                 # max(10, 20) ms / 5 steps
        assert value == pytest.approx(2 * 1000 / 0.004)      # both ranks' units
        assert e2e == pytest.approx(4.0)
