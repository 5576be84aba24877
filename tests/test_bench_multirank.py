"""Host logic of the multi-GPU benchmark path on CPU: two gloo ranks, barrier, max-over-ranks step
time, whole-job throughput = units of all ranks / slowest rank's time; the reference arm runs on
rank 0 only."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    step_ms = 2.0 + rank  # rank 1 is slower
    worst = bench.max_over_ranks(step_ms, world)
    units_per_rank = 1000
    value = units_per_rank * world / (worst * 1e-3)
    out[rank] = (worst, value)
    dist.destroy_process_group()


def test_two_rank_timing_logic():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 3.0
    assert abs(res[0][1] - 2000 / 3e-3) < 1e-6


def test_reference_arm_other_ranks_do_no_work():
    import argparse

    import bench
    args = argparse.Namespace(steps=1, warmup=3)
    assert bench.reference_arm(args, rank=1, world=2) is None
