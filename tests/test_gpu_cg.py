"""GPU Jacobi-PCG on cell-wise data (Sec. 4.4; Eq. (jacobi_recap)) and FP64 iterative refinement
around an FP32 / BF16-metric inner CG, checked against the oracle's assembled PCG and direct solve."""
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


def make(cw, mesh, p, kind=1, geom=None):
    M = cw.Mesh.from_synth(mesh)
    geom = cw.CW_GEOM_METRIC if geom is None else geom
    return M, cw.Operator(M, p, kind, geom, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)


@pytest.mark.parametrize("kind", [1, 3])
@pytest.mark.parametrize("p", [1, 2, 4])
def test_iterates_equal_assembled_pcg(cw, orc, p, kind):
    """Primal-dual CG with the consistent preconditioner D^-1 S is iterate-identical to Jacobi-PCG
    on the assembled interior system (Sec. 4.4)."""
    import torch
    mesh = synth.box_mesh(3, 4, 3, perturb=0.2)
    M, op = make(cw, mesh, p, kind)
    b = orc.load_vector(mesh, p, orc.PROBLEM_SINE)
    A = orc.assemble_global(mesh, p, kind)
    bg = orc.scatter_add(mesh, p, b)
    mask = orc.boundary_mask_global(mesh, p)
    _, _, _, its = orc.pcg_assembled(A, bg, mask, tol=1e-30, maxit=6, record=True)
    bd = torch.from_numpy(b).cuda()
    for k in (1, 3, 6):
        u, st, rc = op.cg_solve(bd, rtol=1e-30, maxit=k, check=False)
        assert rc == cw.CW_ERR_NOT_CONVERGED and st.iterations == k
        assert rel_err(to_np(u), orc.gather(mesh, p, its[k])) <= 1e-10


@pytest.mark.parametrize("p,perturb", [(2, 0.2), (3, 0.0)])
def test_converges_to_direct_solve(cw, orc, p, perturb):
    import torch
    mesh = synth.box_mesh(4, 3, 5, perturb=perturb)
    M, op = make(cw, mesh, p)
    b = orc.load_vector(mesh, p, orc.PROBLEM_SINE)
    A = orc.assemble_global(mesh, p, 1)
    ud = orc.direct_solve(A, orc.scatter_add(mesh, p, b), orc.boundary_mask_global(mesh, p))
    u, st, rc = op.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-12, maxit=2000)
    assert st.rel_residual <= 1e-12
    assert rel_err(to_np(u), orc.gather(mesh, p, ud)) <= 1e-10
    # energy measure eta(u) = <b - A u, u> vanishes at the discrete solution (Eq. (energy_measure))
    assert abs(st.energy) <= 1e-10 * abs(float(b @ orc.gather(mesh, p, ud)))


def test_bubble_is_reproduced(cw, orc):
    """u = x(1-x)y(1-y)z(1-z) is in Q_2: the solve returns its interpolant (affine mesh, Cartesian
    operator)."""
    import torch
    p = 2
    mesh = synth.box_mesh(3, 4, 2)
    M, op = make(cw, mesh, p, geom=cw.CW_GEOM_AFFINE)
    b = op.load_vector(which=1)
    u, st, rc = op.cg_solve(b, rtol=1e-13, maxit=500)
    xyz = orc.node_coords(mesh, p)
    assert np.abs(to_np(u) - np.prod(xyz * (1 - xyz), axis=1)).max() < 1e-11


@pytest.mark.parametrize("mode", [1, 2, 3], ids=["ir_f32", "ir_bf16metric", "f64_native"])
def test_iterative_refinement_reaches_fp64_accuracy(cw, orc, mode):
    import torch
    p = 3
    mesh = synth.box_mesh(6, 5, 4, perturb=0.1)
    M, op = make(cw, mesh, p)
    b = op.load_vector(which=0)
    u64, s64, _ = op.cg_solve(b, rtol=1e-10, maxit=5000, mode=cw.CW_CG_F64)
    uir, sir, _ = op.cg_solve(b, rtol=1e-10, maxit=5000, mode=mode)
    print(f"fp64: {s64.iterations} it {s64.seconds*1e3:.2f} ms res {s64.rel_residual:.2e}; "
          f"ir mode {mode}: {sir.iterations} it in {sir.outer_iterations} outer, res {sir.rel_residual:.2e}")
    assert s64.rel_residual <= 1e-10 and sir.rel_residual <= 1e-10
    if mode != cw.CW_CG_F64_NATIVE:
        assert sir.outer_iterations >= 2
    assert rel_err(to_np(uir), to_np(u64)) <= 1e-8


@pytest.mark.parametrize("mode", [0, 1], ids=["f64", "ir_f32"])
def test_recomputed_geometry_solve(cw, orc, mode):
    """The solver on an operator whose metric is recomputed at the quadrature points: the first
    iterates equal the assembled PCG's, and the converged solution equals the stored-metric one."""
    import torch
    p = 3
    mesh = synth.box_mesh(5, 4, 3, perturb=0.15)
    M, op = make(cw, mesh, p, geom=cw.CW_GEOM_RECOMPUTE)
    _, op_s = make(cw, mesh, p)
    b = op.load_vector(which=0)
    if mode == 0:
        A = orc.assemble_global(mesh, p, 1)
        _, _, _, its = orc.pcg_assembled(A, orc.scatter_add(mesh, p, to_np(b)), orc.boundary_mask_global(mesh, p),
                                         tol=1e-30, maxit=4, record=True)
        u, st, rc = op.cg_solve(b, rtol=1e-30, maxit=4, mode=mode, check=False)
        assert rel_err(to_np(u), orc.gather(mesh, p, its[4])) <= 1e-10
    u, st, _ = op.cg_solve(b, rtol=1e-10, maxit=5000, mode=mode)
    us, ss, _ = op_s.cg_solve(b, rtol=1e-10, maxit=5000, mode=mode)
    assert st.rel_residual <= 1e-10 and ss.rel_residual <= 1e-10
    assert rel_err(to_np(u), to_np(us)) <= 1e-8


def test_discretisation_error_matches_oracle(cw, orc):
    import torch
    p = 2
    mesh = synth.box_mesh(6, perturb=0.1)
    M, op = make(cw, mesh, p)
    b = torch.from_numpy(orc.load_vector(mesh, p)).cuda()
    u, st, rc = op.cg_solve(b, rtol=1e-12, maxit=3000)
    A = orc.assemble_global(mesh, p, 1)
    ud = orc.direct_solve(A, orc.scatter_add(mesh, p, orc.load_vector(mesh, p)), orc.boundary_mask_global(mesh, p))
    e_gpu = orc.error_norms(mesh, p, to_np(u))
    e_ref = orc.error_norms(mesh, p, orc.gather(mesh, p, ud))
    assert abs(e_gpu[0] - e_ref[0]) <= 1e-8 * e_ref[0] and abs(e_gpu[1] - e_ref[1]) <= 1e-8 * e_ref[1]


def test_failures_are_reported_not_raised_on_device(cw):
    """Host-injected failures: a NaN right-hand side ends the solve with CW_ERR_BREAKDOWN (the
    device detects the non-finite scalar and stops the iteration); bad arguments are rejected on
    the host before any launch."""
    import torch
    p = 2
    mesh = synth.box_mesh(3, perturb=0.1)
    M, op = make(cw, mesh, p)
    for idx in (5, 27 * 13 + 13):  # a boundary copy and an interior entry
        b = op.load_vector(0)
        b[idx] = float("nan")
        u, st, rc = op.cg_solve(b, rtol=1e-10, maxit=100, check=False)
        assert rc == cw.CW_ERR_BREAKDOWN, (idx, rc)
    b = op.load_vector(0)
    u = torch.empty_like(b)
    assert cw.load().cw_cg_solve(op.handle, cw._ptr(b), cw._ptr(u), -1.0, 10, 0, None, None) == cw.CW_ERR_ARG
    op32 = cw.Operator(M, p, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F32, cw.CW_BC_DIRICHLET0)
    assert cw.load().cw_cg_solve(op32.handle, cw._ptr(b), cw._ptr(u), 1e-8, 10, 0, None, None) == cw.CW_ERR_ARG
    # the context is still usable
    u, st, rc = op.cg_solve(op.load_vector(0), rtol=1e-10, maxit=500)
    assert st.rel_residual <= 1e-10


@pytest.mark.parametrize("mode", [0, 1, 2, 3], ids=["f64", "ir_f32", "ir_bf16", "f64_native"])
def test_zero_right_hand_side(cw, mode):
    """b = 0: every mode returns u = 0 at once (zero iterations, relative residual 0, CW_OK)."""
    import torch
    mesh = synth.box_mesh(3, 2, 4, perturb=0.1)
    M, op = make(cw, mesh, 2)
    b = torch.zeros(op.L, dtype=torch.float64, device="cuda")
    u = torch.full_like(b, float("nan"))
    u, st, rc = op.cg_solve(b, u, rtol=1e-10, mode=mode)
    assert rc == cw.CW_OK and st.iterations == 0 and st.rel_residual == 0.0
    assert torch.count_nonzero(u).item() == 0


def test_meshes_with_no_and_one_interior_dof(cw, orc):
    """One cell with homogeneous Dirichlet conditions: at p = 1 every DoF is on the boundary (the masked
    right-hand side vanishes; u = 0 with no iteration); at p = 2 the centre node is the only unknown, so
    one CG iteration reaches the oracle's direct solve."""
    import torch
    mesh = synth.box_mesh(1, perturb=0.0)
    M, op = make(cw, mesh, 1)
    b = op.load_vector(0)
    assert torch.count_nonzero(b).item() > 0  # the raw load vector is not zero; its interior part is
    u, st, rc = op.cg_solve(b, rtol=1e-12)
    assert rc == cw.CW_OK and st.iterations == 0 and torch.count_nonzero(u).item() == 0
    mesh2 = synth.box_mesh(1, perturb=0.0)
    M2, op2 = make(cw, mesh2, 2)
    b2 = orc.load_vector(mesh2, 2, orc.PROBLEM_SINE)
    u2, st2, rc2 = op2.cg_solve(torch.from_numpy(b2).cuda(), rtol=1e-12)
    A = orc.assemble_global(mesh2, 2, 1)
    ud = orc.gather(mesh2, 2, orc.direct_solve(A, orc.scatter_add(mesh2, 2, b2), orc.boundary_mask_global(mesh2, 2)))
    assert rc2 == cw.CW_OK and st2.iterations == 1
    assert rel_err(to_np(u2), ud) <= 1e-12


def test_zero_right_hand_side_multigrid_and_multiblock(cw):
    """b = 0 through the multigrid-preconditioned CG and the multi-block CG: u = 0, CW_OK, no iteration."""
    import torch
    ms = [synth.box_mesh(2, perturb=0.1)]
    ms.append(synth.refine(ms[0]))
    ops = [cw.Operator(cw.Mesh.from_synth(m), 2, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
           for m in ms]
    mg = cw.Multigrid(ops)
    b = torch.zeros(ops[-1].L, dtype=torch.float64, device="cuda")
    u, st, rc = mg.pcg_solve(ops[-1], b)
    assert rc == cw.CW_OK and st.iterations == 0 and torch.count_nonzero(u).item() == 0
    mbm = synth.cube_blocks(2, 1, perturb=0.0, seed=1)
    bops = [cw.Operator(cw.Mesh.from_synth(m), 2, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
            for m in mbm.blocks]
    mb = cw.MultiBlock(bops)
    bz = torch.zeros(mb.L, dtype=torch.float64, device="cuda")
    u, st, rc = mb.cg_solve(bz)
    assert rc == cw.CW_OK and st.iterations == 0 and torch.count_nonzero(u).item() == 0


@pytest.mark.parametrize("mode", [0, 1, 2, 3], ids=["f64", "ir_f32", "ir_bf16", "f64_native"])
def test_warm_start_resumes_a_solve(cw, orc, mode):
    """Checkpoint / resume: a solve stopped at rtol 1e-4, copied to the host and back, then continued
    with CW_CG_WARM_START reaches the oracle's direct solve; the residual stays relative to b, a
    converged iterate resumes with no iteration and comes back unchanged, a non-finite iterate is
    reported (CW_ERR_BREAKDOWN) before any write to u, and b = 0 returns u = 0."""
    import torch
    p = 3
    mesh = synth.box_mesh(4, 3, 5, perturb=0.2)
    M, op = make(cw, mesh, p)
    bh = orc.load_vector(mesh, p, orc.PROBLEM_SINE)
    b = torch.from_numpy(bh).cuda()
    A = orc.assemble_global(mesh, p, 1)
    ud = orc.gather(mesh, p, orc.direct_solve(A, orc.scatter_add(mesh, p, bh), orc.boundary_mask_global(mesh, p)))
    u1, s1, rc1 = op.cg_solve(b, rtol=1e-4, maxit=2000, mode=mode)
    assert rc1 == cw.CW_OK and 1e-9 < s1.rel_residual <= 1e-4
    ckpt = to_np(u1).copy()  # the checkpoint lives on the host
    u2 = torch.from_numpy(ckpt).cuda()
    u2, s2, rc2 = op.cg_solve(b, u2, rtol=1e-11, maxit=2000, mode=mode, warm_start=True)
    assert rc2 == cw.CW_OK and s2.rel_residual <= 1e-11 and s2.iterations > 0
    assert rel_err(to_np(u2), ud) <= 1e-9
    assert abs(op.residual(b, u2) - s2.rel_residual) <= 1e-3 * s2.rel_residual
    # resuming from the converged iterate: nothing left to do, u untouched
    keep = u2.clone()
    u3, s3, rc3 = op.cg_solve(b, u2, rtol=1e-10, maxit=2000, mode=mode, warm_start=True)
    assert rc3 == cw.CW_OK and s3.iterations == 0 and s3.outer_iterations == 0
    assert torch.equal(u3, keep)
    # a non-finite iterate is refused before the solve writes u
    bad = torch.from_numpy(ckpt).cuda()
    bad[1 + 4 + 16] = float("nan")  # node (1,1,1) of cell 0: an interior DoF
    bad_in = bad.clone()
    _, _, rc4 = op.cg_solve(b, bad, rtol=1e-10, maxit=100, mode=mode, check=False, warm_start=True)
    assert rc4 == cw.CW_ERR_BREAKDOWN
    assert torch.equal(torch.isnan(bad), torch.isnan(bad_in)) and torch.equal(bad.nan_to_num(), bad_in.nan_to_num())
    # b = 0 with a warm start: the solution is 0 whatever the guess
    u5 = torch.from_numpy(ckpt).cuda()
    u5, s5, rc5 = op.cg_solve(torch.zeros_like(b), u5, rtol=1e-10, mode=mode, warm_start=True)
    assert rc5 == cw.CW_OK and s5.iterations == 0 and torch.count_nonzero(u5).item() == 0
    # an unknown flag bit is an argument error
    assert cw.load().cw_cg_solve(op.handle, cw._ptr(b), cw._ptr(u5), 1e-8, 10, mode | 0x200, None, None) == cw.CW_ERR_ARG
