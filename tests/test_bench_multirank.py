"""The N > 1 benchmark path on CPU: two gloo ranks use bench.py's timing
helpers -- barrier, max over ranks, whole-job rate -- and per-rank seeds."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    from paper_2006_06281_gb300 import datagen
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    barrier, allmax = bench.timing_helpers(world, torch.device("cpu"))
    barrier()
    local_ms = 100.0 * (rank + 1)            # rank 1 is the slower one
    mx = allmax(local_ms)
    cfg = datagen.WORKLOADS["fp64_m500"]
    seed = bench.rank_seed(cfg, rank)
    x0 = float(datagen.gen(16, seed=seed).X[0, 0])
    out[rank] = (mx, bench.job_rate(50, world, mx), seed, x0)
    barrier()
    dist.destroy_process_group()


def test_two_ranks_time_with_the_slowest_and_register_different_pairs():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 200.0           # max over ranks
    assert res[0][1] == pytest.approx(2 * 50 / 0.2)   # all ranks' steps / slowest time
    assert res[0][2] != res[1][2] and res[0][3] != res[1][3]
