"""Failure detection without a GPU fault: the operator kernels' bounded waits for their staged tiles.
A test-only hook arms each staged input tile's barrier with more bytes than its copy delivers, so the
copy lands but the barrier phase never completes and the short bounded wait runs out. The threads must
not read the staged tile (they take zeros), the event must be reported as CW_ERR_TIMEOUT by the next
check or synchronising call (the outputs of that call are undefined), tiles read without staging must
be unaffected, and the context must stay usable."""
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


@pytest.mark.parametrize("prec", [0, 2], ids=["f64", "f32"])
@pytest.mark.parametrize("stage", [1, 2])
def test_expired_wait_is_reported_and_the_context_survives(cw, orc, prec, stage):
    import torch
    p, kind = 2, 3
    probe = cw.Operator(cw.Mesh.from_synth(synth.box_mesh(2, 2, 2)), p, kind, cw.CW_GEOM_METRIC, prec)
    T = probe.variant()[2][0]  # cells per tile of the default variant (16 or 32 at p = 2)
    probe.close()
    mesh = synth.box_mesh(4, 3, T // 8, perturb=0.1)  # 1.5 T cells: one full (staged) tile, one ragged
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, p, kind, cw.CW_GEOM_METRIC, prec)
    op.set_variant(0, stage)
    ug = synth.global_vector(mesh, p, seed=1)
    x = op.gather(torch.from_numpy(ug).cuda())
    ref = orc.apply_local(mesh, p, kind, orc.gather(mesh, p, ug)).reshape(mesh.ncells, -1)
    n3 = (p + 1) ** 3
    cw.cw_op_inject_stall(op.handle, True)
    y = torch.full_like(x, float("nan"))
    cw.cw_apply(op.handle, x, y)
    assert cw.cw_op_check(op.handle) == cw.CW_ERR_TIMEOUT
    assert cw.cw_op_check(op.handle) == cw.CW_OK  # the check clears the word
    yn = to_np(y).reshape(mesh.ncells, n3)
    # the staged tile computed on zeros instead of its unconfirmed input: finite, and not the result
    assert np.isfinite(yn[:T]).all() and rel_err(yn[:T], ref[:T]) > 0.5
    assert rel_err(yn[T:], ref[T:]) <= (1e-12 if prec == 0 else 1e-5)  # the ragged tile reads directly
    cw.cw_op_inject_stall(op.handle, False)
    y2 = op.apply(x)
    assert cw.cw_op_check(op.handle) == cw.CW_OK
    assert rel_err(to_np(y2).reshape(mesh.ncells, n3), ref) <= (1e-12 if prec == 0 else 1e-5)


def test_synchronising_calls_report_the_timeout(cw, orc):
    """The solver's operator (the <p, Ap> kernel, TMA-staged) and a multigrid level: the solve returns
    CW_ERR_TIMEOUT; disarmed, the same handles solve normally."""
    import torch
    p = 2
    m0 = synth.box_mesh(2, perturb=0.1)
    ms = [m0, synth.refine(m0), synth.refine(synth.refine(m0))]
    Ms = [cw.Mesh.from_synth(m) for m in ms]
    op = cw.Operator(Ms[-1], p, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
    b = op.load_vector(0)
    cw.cw_op_inject_stall(op.handle, True)
    u, st, rc = op.cg_solve(b, rtol=1e-10, maxit=200, check=False)
    assert rc == cw.CW_ERR_TIMEOUT
    cw.cw_op_inject_stall(op.handle, False)
    u, st, rc = op.cg_solve(b, rtol=1e-10, maxit=2000)
    assert rc == cw.CW_OK and st.rel_residual <= 1e-10
    ops = [cw.Operator(M, p, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F32, cw.CW_BC_DIRICHLET0) for M in Ms]
    mg = cw.Multigrid(ops)
    cw.cw_op_inject_stall(ops[-1].handle, True)
    u, st, rc = mg.pcg_solve(op, b, rtol=1e-10, maxit=100, check=False)
    assert rc == cw.CW_ERR_TIMEOUT
    cw.cw_op_inject_stall(ops[-1].handle, False)
    u, st, rc = mg.pcg_solve(op, b, rtol=1e-10, maxit=100)
    assert rc == cw.CW_OK and st.rel_residual <= 1e-10
