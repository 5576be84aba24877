"""The allocation-free solver entry point, cw_cg_solve_noalloc, for callers that must not allocate
device memory while solving (code inside a memory pool or allocator callback, real-time loops with
memory fixed at start-up). It must give the same solution as cw_cg_solve on consecutive calls
that share its fixed scratch array, allocate nothing itself, and reject operators beyond its size
limit. This file is collected last so that a stop at the first failure has already run every other
test."""
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


@pytest.mark.parametrize("mode", [0, 3], ids=["f64_doublefloat", "f64_native"])
def test_noalloc_matches_cg_solve_on_two_calls(cw, mode):
    import torch
    p = 3
    mesh = synth.box_mesh(6, 5, 4, perturb=0.1)
    M = cw.Mesh.from_synth(mesh)
    # a fresh operator that never sees cw_cg_solve: no solver scratch exists for it, so the entry
    # point cannot lean on scratch made by another call
    op = cw.Operator(M, p, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
    op_ref = cw.Operator(M, p, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
    b = op.load_vector(0)
    us = [torch.full_like(b, float("nan")) for _ in range(2)]  # every entry must be written
    uk = [torch.empty_like(b) for _ in range(2)]
    torch.cuda.synchronize()
    bytes0 = cw.cw_op_device_bytes(op.handle)
    free = []
    for call in range(2):
        rc, st = cw.cw_cg_solve_noalloc(op.handle, b, us[call], 1e-10, 5000, mode)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert rc == cw.CW_OK, (call, cw.load().cw_last_error())
        assert st.rel_residual <= 1e-10
    for call in range(2):
        rc, st = cw.cw_cg_solve_noalloc(op.handle, b, uk[call], 1e-30, 7, mode)
        torch.cuda.synchronize()
        assert rc == cw.CW_ERR_NOT_CONVERGED and st.iterations == 7
    # nothing was allocated: the operator owns what it owned before, and the device's free memory did
    # not move between the first and the second call
    assert cw.cw_op_device_bytes(op.handle) == bytes0
    assert free[1] == free[0]
    u_ref, st_ref, rc = op_ref.cg_solve(b, rtol=1e-10, maxit=5000, mode=mode)
    assert st_ref.rel_residual <= 1e-10
    for call in range(2):
        assert rel_err(to_np(us[call]), to_np(u_ref)) <= 1e-8, call
    # fixed iteration count: the iterates themselves agree
    u_k, _, _ = op_ref.cg_solve(b, rtol=1e-30, maxit=7, mode=mode, check=False)
    for call in range(2):
        assert rel_err(to_np(uk[call]), to_np(u_k)) <= 1e-10, call


def test_noalloc_rejects_operators_beyond_its_limit(cw):
    import torch
    mesh = synth.box_mesh(18, perturb=0.1)  # 5832 cells x 64 = 373,248 values > 2^18
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, 3, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
    b = torch.zeros(op.L, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(b)
    rc, st = cw.cw_cg_solve_noalloc(op.handle, b, u, 1e-10, 10, 0)
    assert rc == cw.CW_ERR_ARG
    assert b"262144" in cw.load().cw_last_error()


def test_noalloc_always_starts_from_zero(cw):
    """The allocation-free solve has no warm start: CW_CG_WARM_START is an argument error there."""
    import torch
    M = cw.Mesh.from_synth(synth.box_mesh(3, perturb=0.1))
    op = cw.Operator(M, 2, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
    b = op.load_vector(0)
    u = torch.zeros_like(b)
    rc, st = cw.cw_cg_solve_noalloc(op.handle, b, u, 1e-10, 10, cw.CW_CG_F64 | cw.CW_CG_WARM_START)
    assert rc == cw.CW_ERR_ARG
