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
    with mp.get_context("spawn").Manager() as m:  # no fork of a multi-threaded parent
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


def test_reference_arm_json_contract():
    """Rank 0 of the reference arm times the oracle on the host cores and returns the contract's
    line: the base keys, "impl": "reference", a cpu_baseline describing the run and an e2e entry
    with no host-device bytes."""
    import argparse
    import json

    import bench
    r = bench.reference_arm(argparse.Namespace(steps=1, warmup=3), rank=0, world=1)
    json.dumps(r)  # serialisable as one line
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in r, k
    assert r["impl"] == "reference" and r["value"] > 0 and r["steps"] == 1 and r["warmup"] == 3
    assert r["higher_is_better"] is True and r["vs_baseline"] is None and "workload" in r["config"]
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == r["value"] and cb["cores"] >= 1 and cb["sample"]
    e = r["e2e"]
    assert e["value"] == r["value"] and e["unit"] == r["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
