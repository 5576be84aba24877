"""Every solver mode against the oracle (Sec. 4.4: the cell-wise primal-dual CG solves the assembled
system; the refined modes keep FP64 for the outer residual). The solution is compared with the
oracle's sparse direct solve, and its residual is recomputed with the oracle's assembled A_CG
(explicit element matrices, brute-force assembly), independently of the library's operators."""
import numpy as np
import pytest

import synth
from gpu_util import rel_err, to_np

pytestmark = pytest.mark.gpu

MODES = {"f64_doublefloat": 0, "ir_f32": 1, "ir_bf16metric": 2, "f64_native": 3}


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


def oracle_residual(orc, mesh, p, A, bg, mask, u_cell):
    """||m (G^T b - A_CG u_g)|| / ||m G^T b|| with u_g the average of the copies of each DoF."""
    ones = np.ones_like(u_cell)
    ug = orc.scatter_add(mesh, p, u_cell) / orc.scatter_add(mesh, p, ones)
    return float(np.linalg.norm(mask * (bg - A @ ug)) / np.linalg.norm(mask * bg))


@pytest.mark.parametrize("mode", list(MODES.values()), ids=list(MODES))
@pytest.mark.parametrize("shape,p", [((4, 3, 5), 2), ((4, 3, 5), 3), ((8, 8, 8), 2)])
def test_solution_matches_oracle_direct_solve(cw, orc, mode, shape, p):
    import torch
    mesh = synth.box_mesh(*shape, perturb=0.1)
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, p, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
    b = orc.load_vector(mesh, p, orc.PROBLEM_SINE)
    A = orc.assemble_global(mesh, p, 1)
    bg = orc.scatter_add(mesh, p, b)
    mask = orc.boundary_mask_global(mesh, p)
    ud = orc.gather(mesh, p, orc.direct_solve(A, bg, mask))
    u, st, rc = op.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-13, maxit=20000, mode=mode)
    un = to_np(u)
    res = oracle_residual(orc, mesh, p, A, bg, mask, un)
    err = rel_err(un, ud)
    print(f"mode {mode} {shape} p={p}: {st.iterations} it / {st.outer_iterations} outer, "
          f"library residual {st.rel_residual:.2e}, oracle residual {res:.2e}, error vs direct {err:.2e}")
    assert st.rel_residual <= 1e-13
    assert res <= 1e-10
    assert err <= 1e-10


@pytest.mark.slow
@pytest.mark.parametrize("mode", [1, 2], ids=["ir_f32", "ir_bf16metric"])
def test_refined_solve_at_the_largest_assembled_mesh(cw, orc, mode):
    """16^3 curved cells, Q3 (117,649 global DoFs): the largest mesh the oracle assembles in seconds.
    The refined solve's residual is recomputed with the oracle's A_CG, and its solution compared with
    the oracle's assembled Jacobi-PCG solved to 1e-14."""
    import torch
    p = 3
    mesh = synth.box_mesh(16, perturb=0.1)
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, p, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
    b = orc.load_vector(mesh, p, orc.PROBLEM_SINE)
    A = orc.assemble_global(mesh, p, 1)
    bg = orc.scatter_add(mesh, p, b)
    mask = orc.boundary_mask_global(mesh, p)
    u_or, its, rel_or, _ = orc.pcg_assembled(A, bg, mask, tol=1e-14, maxit=5000)
    assert rel_or <= 1e-14
    # 1e-12: about 100 units of FP64 rounding at this size (the smaller meshes above reach 1e-13)
    u, st, rc = op.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-12, maxit=50000, mode=mode)
    un = to_np(u)
    res = oracle_residual(orc, mesh, p, A, bg, mask, un)
    err = rel_err(un, orc.gather(mesh, p, u_or))
    print(f"16^3 Q3 mode {mode}: {st.iterations} it / {st.outer_iterations} outer, library residual "
          f"{st.rel_residual:.2e}, oracle residual {res:.2e}, error vs oracle PCG {err:.2e}")
    assert res <= 1e-10 and err <= 1e-10
    # the library's two residual measures of the same iterate: the IEEE FP64 operator agrees with the
    # oracle's A_CG to well below the tolerance; double-float on the float-pair metric is reported
    r_ieee = op.residual(torch.from_numpy(b).cuda(), u, cw.CW_PREC_F64_NATIVE)
    r_df = op.residual(torch.from_numpy(b).cuda(), u, cw.CW_PREC_F64)
    print(f"residual of the same iterate: IEEE operator {r_ieee:.3e}, double-float operator {r_df:.3e}")
    assert abs(r_ieee - res) <= 1e-12, (r_ieee, res)
    assert r_df <= 1e-9


def test_native_operator_stores_an_ieee_metric(cw, orc):
    """CW_PREC_F64_NATIVE keeps the metric in IEEE doubles: its apply matches the oracle to a few
    units of FP64 rounding (tighter than the float-pair metric of CW_PREC_F64 allows)."""
    import torch
    p = 3
    mesh = synth.box_mesh(5, 4, 3, perturb=0.15)
    M = cw.Mesh.from_synth(mesh)
    ug = synth.global_vector(mesh, p, seed=3)
    ref = orc.apply_local(mesh, p, 3, orc.gather(mesh, p, ug))
    errs = {}
    for prec in (cw.CW_PREC_F64_NATIVE, cw.CW_PREC_F64):
        for geom in (cw.CW_GEOM_METRIC, cw.CW_GEOM_RECOMPUTE):
            op = cw.Operator(M, p, 3, geom, prec)
            y = op.apply(op.gather(torch.from_numpy(ug).cuda()))
            errs[(prec, geom)] = rel_err(to_np(y), ref)
    print(errs)
    assert errs[(cw.CW_PREC_F64_NATIVE, cw.CW_GEOM_METRIC)] <= 1e-14
    assert errs[(cw.CW_PREC_F64_NATIVE, cw.CW_GEOM_RECOMPUTE)] <= 1e-14
    assert max(errs.values()) <= 1e-12
    # the IEEE twin the solver builds is counted in the operator's device bytes
    op = cw.Operator(M, p, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
    before = cw.cw_op_device_bytes(op.handle)
    op.cg_solve(op.load_vector(0), rtol=1e-6, maxit=100)
    after = cw.cw_op_device_bytes(op.handle)
    metric_bytes = mesh.ncells * 6 * (p + 1) ** 3 * 8
    assert after - before >= metric_bytes
