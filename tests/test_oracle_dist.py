"""The slab-partitioned DSS and Jacobi-PCG of ``oracle.dist`` on gloo ranks (CPU) against the
single-process oracle: the face-layer exchange completes Algorithm struct_dss across ranks, and the
distributed primal-dual CG follows the assembled Jacobi-PCG iterate by iterate."""
import os
import socket

import numpy as np
import pytest

import synth

P = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def mesh_case():
    return synth.box_mesh(3, 2, 5, perturb=0.2)


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from oracle import dist as od
    mesh = mesh_case()
    slab = od.Slab(mesh, rank, world)
    v = synth.cellwise_random(mesh, P, seed=1)
    s_part = od.dss(slab, P, slab.part(v, P))
    b = oracle.load_vector(mesh, P)
    its = od.pcg(slab, P, oracle.KIND_LAPLACE, slab.part(b, P), 5)
    out[rank] = (s_part, np.array(its))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_distributed_dss_and_pcg(orc, world):
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a multi-threaded parent
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    mesh = mesh_case()
    v = synth.cellwise_random(mesh, P, seed=1)
    ref = orc.dss(mesh, P, v)
    got = np.concatenate([res[r][0] for r in range(world)])
    assert np.abs(got - ref).max() < 1e-14 * np.abs(ref).max()
    b = orc.load_vector(mesh, P)
    A = orc.assemble_global(mesh, P, orc.KIND_LAPLACE)
    mask = orc.boundary_mask_global(mesh, P)
    _, _, _, its = orc.pcg_assembled(A, orc.scatter_add(mesh, P, b), mask, tol=1e-30, maxit=5, record=True)
    for k in range(6):
        got = np.concatenate([res[r][1][k] for r in range(world)])
        ref = orc.gather(mesh, P, its[k])
        assert np.abs(got - ref).max() <= 1e-10 * max(np.abs(ref).max(), 1e-300), k


def _lost_rank_main(rank, world, port, out):
    import datetime

    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:  # this rank leaves between steps, before the exchange, without a word
        out[rank] = "left"
        return
    from oracle import dist as od
    mesh = mesh_case()
    slab = od.Slab(mesh, rank, world)
    try:
        od.dss(slab, P, slab.part(synth.cellwise_random(mesh, P, seed=1), P))
        out[rank] = "completed"
    except Exception as e:  # the lost peer surfaces as an error of the exchange, not a hang
        out[rank] = "error: " + type(e).__name__


@pytest.mark.timeout(180)
def test_lost_rank_is_reported_not_hung(orc):
    """Failure detection on the host: a rank that leaves before the face-layer exchange makes its
    neighbour's exchange fail with an error (peer closed, or the process-group timeout)."""
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_lost_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[1] == "left" and res[0].startswith("error"), res
