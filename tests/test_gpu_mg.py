"""GPU geometric multigrid (Sec. 3 and 5) against the oracle's multigrid (oracle.mg): the cell-wise
transfers (Algorithms prolongation and restriction), the fused smoother (Algorithm smoother_fused),
the coarse solve, the V-cycle (Algorithm mg_vcycle) and the V-cycle-preconditioned CG, in the
double-float, IEEE FP64 and FP32 arithmetics."""
import numpy as np
import pytest

import synth
from gpu_util import rel_err, to_np

pytestmark = pytest.mark.gpu

# element-wise bounds against the FP64 oracle per arithmetic (double-float, IEEE FP64, FP32)
TOL = {0: 1e-12, 1: 1e-13, 2: 2e-6}


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


@pytest.fixture(scope="module")
def omg(orc):
    from oracle import mg
    return mg


def meshes(m0, nl):
    ms = [m0]
    for _ in range(nl - 1):
        ms.append(synth.refine(ms[-1]))
    return ms


def gpu_hierarchy(cw, ms, p, prec, kind=1, geom=None, **kw):
    geom = cw.CW_GEOM_METRIC if geom is None else geom
    Ms = [cw.Mesh.from_synth(m) for m in ms]
    ops = [cw.Operator(M, p, kind, geom, prec, cw.CW_BC_DIRICHLET0) for M in Ms]
    return Ms, ops, cw.Multigrid(ops, **kw)


def dev(t, op):
    import torch
    return torch.from_numpy(np.ascontiguousarray(t)).to("cuda", op.vec_dtype)


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["doublefloat", "ieee_f64", "f32"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_transfers_match_oracle(cw, orc, omg, p, prec):
    """Prolongation of a coarse cell-wise vector and restriction of a fine raw dual, element by
    element (odd coarse sizes, curved cells: the transfers only read the hierarchy's numbering)."""
    # the coarse level stays within the dense coarse solve's limit (4096 interior DoFs)
    mc = synth.box_mesh(3, 2, 3, perturb=0.2) if p <= 3 else synth.box_mesh(2, 1, 2, perturb=0.2)
    ms = meshes(mc, 2)
    Ms, ops, mg = gpu_hierarchy(cw, ms, p, prec)
    uc = synth.cellwise_random(mc, p, seed=p)
    rf = synth.cellwise_random(ms[1], p, seed=10 + p)
    uf = to_np(mg.prolong(1, dev(uc, ops[0])))
    rc = to_np(mg.restrict(1, dev(rf, ops[1])))
    if prec == 2:  # the oracle on the FP32-rounded inputs
        uc, rf = uc.astype(np.float32).astype(np.float64), rf.astype(np.float32).astype(np.float64)
    assert rel_err(uf, omg.prolong(mc, p, uc)) <= TOL[prec]
    assert rel_err(rc, omg.restrict(mc, p, rf)) <= TOL[prec]


@pytest.mark.parametrize("p", [1, 3])
def test_transfers_of_a_three_level_cube(cw, orc, omg, p):
    """Level 2 <- 1 <- 0 on the Cartesian cube: a prolonged continuous vector stays continuous (the
    gather commutes with prolongation, Lemma prolongation_commutativity)."""
    ms = meshes(synth.box_mesh(2), 3)
    Ms, ops, mg = gpu_hierarchy(cw, ms, p, 0)
    ug = synth.global_vector(ms[1], p, seed=3)
    u1 = orc.gather(ms[1], p, ug)
    u2 = to_np(mg.prolong(2, dev(u1, ops[1])))
    ref = omg.prolong(ms[1], p, u1)
    assert rel_err(u2, ref) <= 1e-12
    # continuity: the averaging DSS leaves it unchanged
    assert rel_err(orc.dss(ms[2], p, u2) / orc.dss(ms[2], p, np.ones_like(u2)), u2) <= 1e-13


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["doublefloat", "ieee_f64", "f32"])
@pytest.mark.parametrize("p", [2, 3])
def test_coarse_solve_and_smoother_match_oracle(cw, orc, omg, p, prec):
    ms = meshes(synth.box_mesh(2, 3, 2, perturb=0.2), 2)
    Ms, ops, mg = gpu_hierarchy(cw, ms, p, prec)
    lv = omg.hierarchy(ms, p, 1)
    b0 = synth.cellwise_random(ms[0], p, seed=1)
    u0 = to_np(mg.coarse_solve(dev(b0, ops[0])))
    if prec == 2:
        b0 = b0.astype(np.float32).astype(np.float64)
    assert rel_err(u0, omg.coarse_solve(lv[0], b0)) <= (1e-12 if prec < 2 else 1e-5)
    # one and two fused smoothing sweeps on the fine level from a continuous iterate
    m = ms[1]
    u = orc.gather(m, p, synth.global_vector(m, p, seed=2) * lv[1].mask)
    b = synth.cellwise_random(m, p, seed=3)
    for sweeps in (1, 2):
        ud = dev(u, ops[1])
        mg.smooth(1, dev(b, ops[1]), ud, sweeps)
        ref = u.copy()
        for _ in range(sweeps):
            ref = omg.smooth_fused(lv[1], b, ref, 0.7)
        assert rel_err(to_np(ud), ref) <= (TOL[prec] if prec < 2 else 1e-5), sweeps


@pytest.mark.parametrize("prec", [0, 1], ids=["doublefloat", "ieee_f64"])
@pytest.mark.parametrize("p,perturb,geom", [(1, 0.3, 1), (2, 0.3, 1), (3, 0.0, 1), (3, 0.2, 1), (2, 0.3, 2),
                                            (3, 0.0, 0)], ids=["p1", "p2", "p3cart", "p3", "p2recomputed",
                                                               "p3affine"])
def test_vcycle_matches_oracle(cw, orc, omg, p, perturb, geom, prec):
    """One V-cycle on three levels, from zero and from a continuous initial guess, against the
    oracle's cell-wise V-cycle in the fused form (stored and recomputed metric: sweeps fused into the
    operator launch in double-float; Cartesian cells and IEEE FP64: operator, update and averaging
    passes as separate launches)."""
    ms = meshes(synth.box_mesh(2, 3, 2, perturb=perturb), 3)
    Ms, ops, mg = gpu_hierarchy(cw, ms, p, prec, geom=geom)
    lv = omg.hierarchy(ms, p, 1)
    m = ms[2]
    b = synth.cellwise_random(m, p, seed=5)
    z = to_np(mg.vcycle(dev(b, ops[2])))
    ref = omg.vcycle(lv, 2, b, np.zeros_like(b), fused=True)
    assert rel_err(z, ref) <= 1e-11
    u0 = orc.gather(m, p, synth.global_vector(m, p, seed=6) * lv[2].mask)
    ud = dev(u0, ops[2])
    mg.vcycle(dev(b, ops[2]), ud, zero_guess=False)
    assert rel_err(to_np(ud), omg.vcycle(lv, 2, b, u0, fused=True)) <= 1e-11


@pytest.mark.parametrize("p", [2, 3, 5])
def test_fp32_vcycle_matches_oracle_fp32_cycle(cw, orc, omg, p):
    """The FP32 cycle against the oracle's FP32-storage cycle (every vector rounded to FP32 after each
    step, FP64 arithmetic within a step): agreement to FP32 rounding, far from the FP64 result's
    distance to zero."""
    ms = meshes(synth.box_mesh(2, 3, 2, perturb=0.2), 3)
    Ms, ops, mg = gpu_hierarchy(cw, ms, p, 2)
    lv = omg.hierarchy(ms, p, 1)
    b = omg.average(lv[2], synth.cellwise_random(ms[2], p, seed=7))
    z = to_np(mg.vcycle(dev(b, ops[2])))
    ref32 = omg.vcycle(lv, 2, b, np.zeros_like(b), fused=True, dtype=np.float32)
    ref64 = omg.vcycle(lv, 2, b, np.zeros_like(b), fused=True)
    print(f"p={p}: FP32 cycle vs oracle FP32 {rel_err(z, ref32):.2e}, vs oracle FP64 {rel_err(z, ref64):.2e}")
    assert rel_err(z, ref32) <= 2e-5 and rel_err(z, ref64) <= 2e-5


@pytest.mark.parametrize("p", [2, 3])
def test_mg_pcg_iterates_match_oracle(cw, orc, omg, p):
    """The V-cycle-preconditioned CG after k iterations equals the oracle's MG-PCG after k (Sec. 5:
    zero initial guess in the preconditioner; the cycle fed S_bar r, which it reads only through
    G^T, as the raw r the oracle feeds)."""
    import torch
    ms = meshes(synth.box_mesh(2, 2, 3, perturb=0.2), 3)
    Ms, ops, mg = gpu_hierarchy(cw, ms, p, 0)
    fine = cw.Operator(Ms[-1], p, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
    lv = omg.hierarchy(ms, p, 1)
    b = orc.load_vector(ms[-1], p)
    bd = torch.from_numpy(b).cuda()
    for k in (1, 3):
        u, st, rc = mg.pcg_solve(fine, bd, rtol=1e-30, maxit=k, check=False)
        assert rc == cw.CW_ERR_NOT_CONVERGED and st.iterations == k
        ref, kk, _ = omg.mg_pcg(lv, b, tol=0.0, maxit=k, fused=True)
        assert kk == k
        assert rel_err(to_np(u), ref) <= 1e-10, k


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["doublefloat", "ieee_f64", "f32"])
@pytest.mark.parametrize("p,nl", [(2, 3), (3, 3), (4, 2)])
def test_mg_pcg_converges_to_direct_solve(cw, orc, omg, p, nl, prec):
    """Converged MG-PCG: the solution equals the oracle's direct solve, the residual recomputed with
    the oracle's A_CG is below the tolerance, and the iteration count is the handful the paper's
    cube runs show (8-11 for a 1e-14 energy reduction), FP32 cycle included."""
    import torch
    ms = meshes(synth.box_mesh(2, perturb=0.1), nl)
    Ms, ops, mg = gpu_hierarchy(cw, ms, p, prec)
    fine = cw.Operator(Ms[-1], p, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
    m = ms[-1]
    b = orc.load_vector(m, p)
    A = orc.assemble_global(m, p, 1)
    bg, mask = orc.scatter_add(m, p, b), orc.boundary_mask_global(m, p)
    ud = orc.gather(m, p, orc.direct_solve(A, bg, mask))
    u, st, rc = mg.pcg_solve(fine, torch.from_numpy(b).cuda(), rtol=1e-12, maxit=200)
    un = to_np(u)
    ug = orc.scatter_add(m, p, un) / orc.scatter_add(m, p, np.ones_like(un))
    res = np.linalg.norm(mask * (bg - A @ ug)) / np.linalg.norm(mask * bg)
    print(f"p={p} levels={nl} prec={prec}: {st.iterations} it / {st.outer_iterations} outer, "
          f"residual {st.rel_residual:.2e} (oracle {res:.2e}), error {rel_err(un, ud):.2e}")
    assert st.rel_residual <= 1e-12 and res <= 1e-11
    assert rel_err(un, ud) <= 1e-10
    assert st.iterations <= 30


def test_mg_argument_errors(cw):
    import torch
    p = 2
    m0 = synth.box_mesh(3, perturb=0.1)
    m1 = synth.box_mesh(6, perturb=0.1)  # not the refinement of m0: the displacement scales with h
    M0, M1 = cw.Mesh.from_synth(m0), cw.Mesh.from_synth(m1)
    o0 = cw.Operator(M0, p, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
    o1 = cw.Operator(M1, p, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
    L = cw.load()
    VP = __import__("ctypes").c_void_p
    h = VP()
    arr = (VP * 2)(o0.handle.value, o1.handle.value)
    assert L.cw_mg_create(arr, 2, 2, 2, 0.7, __import__("ctypes").byref(h)) == cw.CW_ERR_ARG
    assert b"nested" in L.cw_last_error()
    o1n = cw.Operator(M0, p, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_NONE)
    arr1 = (VP * 1)(o1n.handle.value)
    assert L.cw_mg_create(arr1, 1, 2, 2, 0.7, __import__("ctypes").byref(h)) == cw.CW_ERR_ARG
    # a coarsest level beyond the dense solve's limit
    Mb = cw.Mesh.from_synth(synth.box_mesh(9))
    ob = cw.Operator(Mb, 2, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)  # 17^3 interior DoFs
    arr2 = (VP * 1)(ob.handle.value)
    assert L.cw_mg_create(arr2, 1, 2, 2, 0.7, __import__("ctypes").byref(h)) == cw.CW_ERR_UNSUPPORTED
    mg = cw.Multigrid([o0])
    fine_other = cw.Operator(M1, p, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
    b = torch.zeros(fine_other.L, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(b)
    rc, st = cw.cw_mg_pcg_solve(mg.handle, fine_other.handle, b, u, check=False)
    assert rc == cw.CW_ERR_ARG
