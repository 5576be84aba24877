"""Batched apply: many operators (uneven meshes, mixed degrees, several right-hand sides) in one
persistent launch, plain or replayed from a CUDA graph, against the per-operator apply and the
oracle."""
import numpy as np
import pytest

import synth
from gpu_util import rel_err, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_03413_gb300 as cw
    from paper_2607_03413_gb300 import build
    build.build()
    cw.load()
    return cw


def make_batch(cw, prec, specs):
    import torch
    meshes, ops, xs, ys, nrhs, refs = [], [], [], [], [], []
    for i, (n, p, R, kind) in enumerate(specs):
        m = synth.box_mesh(n, n + 1, max(1, n - 1), perturb=0.15, freq=(1 + i % 3, 2, 1 + i % 2))
        M = cw.Mesh.from_synth(m)
        op = cw.Operator(M, p, kind, cw.CW_GEOM_METRIC, prec)
        x = torch.stack([op.gather(torch.from_numpy(synth.global_vector(m, p, seed=10 * i + r)).cuda())
                         for r in range(R)]).contiguous()
        y = torch.full_like(x, float("nan"))
        meshes.append((m, M))
        ops.append(op)
        xs.append(x)
        ys.append(y)
        nrhs.append(R)
    return meshes, ops, xs, ys, nrhs


SPECS = [(3, 2, 2, 1), (4, 3, 1, 3), (2, 5, 3, 1), (3, 7, 1, 2), (5, 1, 1, 1), (2, 4, 2, 3), (3, 6, 1, 1)]


@pytest.mark.parametrize("mode", [0, 1], ids=["grouped", "single"])
@pytest.mark.parametrize("prec", [0, 2], ids=["df64", "f32"])
@pytest.mark.parametrize("graph", [False, True])
def test_batch_equals_per_operator_apply(cw, prec, graph, mode):
    import torch
    meshes, ops, xs, ys, nrhs = make_batch(cw, prec, SPECS)
    B = cw.Batch(ops, nrhs, xs, ys)
    B.set_mode(mode)
    assert B.values == sum(o.L * r for o, r in zip(ops, nrhs))
    for variant in range(6 if mode == 0 else 2):
        for (_, p, _, _) in SPECS:
            B.set_variant(p, variant)
        for y in ys:
            y.fill_(float("nan"))
        B.launch(graph=graph)
        B.launch(graph=graph)  # a second launch (graph replay) gives the same result
        torch.cuda.synchronize()
        for op, x, y, R in zip(ops, xs, ys, nrhs):
            for r in range(R):
                ref = op.apply(x[r])
                torch.cuda.synchronize()
                if prec == 0:  # same double-float operation sequence per cell: bit-identical
                    assert torch.equal(y[r], ref)
                else:
                    assert rel_err(to_np(y[r]), to_np(ref)) <= 1e-6
    B.close()


@pytest.mark.parametrize("mode", [0, 1], ids=["grouped", "single"])
def test_batch_matches_oracle_and_autotunes(cw, orc, mode):
    import torch
    meshes, ops, xs, ys, nrhs = make_batch(cw, 0, SPECS)
    B = cw.Batch(ops, nrhs, xs, ys)
    B.set_mode(mode)
    ms = B.autotune(reps=2)
    assert ms > 0
    B.launch(graph=True)
    torch.cuda.synchronize()
    for (m, _), op, x, y, R, (n, p, _, kind) in zip(meshes, ops, xs, ys, nrhs, SPECS):
        r = R - 1
        ref = orc.apply_local(m, p, kind, to_np(x[r]))
        assert rel_err(to_np(y[r]), ref) <= 1e-12, (n, p)


@pytest.mark.parametrize("prec", [0, 2], ids=["df64", "f32"])
def test_apply_batched_one_shot(cw, orc, prec):
    """cw_apply_batched: LOCAL equals a launch of a kept batch; ASSEMBLE equals the oracle's S A x."""
    import torch
    meshes, ops, xs, ys, nrhs = make_batch(cw, prec, SPECS)
    B = cw.Batch(ops, nrhs, xs, ys)
    B.launch()
    torch.cuda.synchronize()
    kept = [y.clone() for y in ys]
    B.close()
    handles = [o.handle for o in ops]
    for y in ys:
        y.fill_(float("nan"))
    cw.cw_apply_batched(handles, xs, ys, nrhs, cw.CW_APPLY_LOCAL)
    for y, k in zip(ys, kept):
        assert torch.equal(y, k)
    for y in ys:
        y.fill_(float("nan"))
    cw.cw_apply_batched(handles, xs, ys, nrhs, cw.CW_APPLY_ASSEMBLE)
    tol = 1e-12 if prec == 0 else 1e-5
    for (m, _), x, y, R, (n, p, _, kind) in zip(meshes, xs, ys, nrhs, SPECS):
        for r in range(R):
            ref = orc.dss(m, p, orc.apply_local(m, p, kind, to_np(x[r])))
            assert rel_err(to_np(y[r]), ref) <= tol, (n, p, r)
    with pytest.raises(cw.CwError):  # flags outside LOCAL / ASSEMBLE
        cw.cw_apply_batched(handles, xs, ys, nrhs, 7)


def test_batch_argument_errors(cw):
    import torch
    m = synth.box_mesh(2, perturb=0.1)
    M = cw.Mesh.from_synth(m)
    op16 = cw.Operator(M, 2, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_BF16)
    x = op16.empty()
    y = op16.empty()
    with pytest.raises(cw.CwError):
        cw.Batch([op16], [1], [x], [y])
    op64 = cw.Operator(M, 2, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64)
    op32 = cw.Operator(M, 2, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F32)
    with pytest.raises(cw.CwError):  # mixed precisions
        cw.Batch([op64, op32], [1, 1], [op64.empty(), op32.empty()], [op64.empty(), op32.empty()])
