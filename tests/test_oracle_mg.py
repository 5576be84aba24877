"""Pins for the oracle's geometric multigrid of a uniform mesh hierarchy (Sec. 3-5): the cell-wise
transfers against closed forms, polynomial reproduction and the classical global prolongation
built another way; the smoother's literal and fused forms against the assembled damped Jacobi;
the cell-wise V-cycle against the classical V-cycle; and the V-cycle-preconditioned CG."""
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def mg(orc):
    from oracle import mg as m
    return m


def test_prolongation_1d_closed_forms(mg):
    data = [list(map(float, ln.split())) for ln in open(os.path.join(GOLDEN, "prolong_1d.txt"))
            if ln.strip() and not ln.startswith("#")]
    for r in data:
        p, b, i = int(r[0]), int(r[1]), int(r[2])
        P = mg.prolongation_1d(p)[b]
        assert np.abs(P[i] - np.array(r[3:])).max() < 1e-15, (p, b, i)


@pytest.mark.parametrize("p", range(1, 8))
def test_prolongation_1d_properties(mg, orc, p):
    P0, P1 = mg.prolongation_1d(p)
    xi = orc.gll(p)
    J = np.eye(p + 1)[::-1]
    assert np.abs(P0.sum(axis=1) - 1).max() < 1e-13 and np.abs(P1.sum(axis=1) - 1).max() < 1e-13
    for k in range(p + 1):  # degree-p polynomials are reproduced exactly (nested spaces)
        for b, P in ((0, P0), (1, P1)):
            assert np.abs(P @ xi ** k - ((xi + b) / 2) ** k).max() < 1e-13, (k, b)
    assert np.abs(P1 - J @ P0 @ J).max() < 1e-13  # reflection x -> 1 - x swaps the children
    assert np.abs(P0[-1] - P1[0]).max() < 1e-15   # the shared midpoint node


def test_refine_closed_forms():
    assert np.abs(synth.refine(synth.box_mesh(3, 2, 4)).verts - synth.box_mesh(6, 4, 8).verts).max() < 1e-15
    c = synth.box_mesh(3, perturb=0.3)
    f = synth.refine(c)
    V, W = c.verts, f.verts
    assert (f.nx, f.ny, f.nz) == (6, 6, 6) and np.array_equal(W[::2, ::2, ::2], V)
    # the trilinear map at the half points: edge midpoints, face centres and cell centres are the
    # averages of the 2, 4 and 8 parent vertices
    assert np.abs(W[::2, ::2, 1::2] - 0.5 * (V[:, :, :-1] + V[:, :, 1:])).max() < 1e-15
    face = 0.25 * (V[:, :-1, :-1] + V[:, :-1, 1:] + V[:, 1:, :-1] + V[:, 1:, 1:])
    assert np.abs(W[::2, 1::2, 1::2] - face).max() < 1e-15
    cell = sum(V[a:a + 3, b:b + 3, d:d + 3] for a in (0, 1) for b in (0, 1) for d in (0, 1)) / 8
    assert np.abs(W[1::2, 1::2, 1::2] - cell).max() < 1e-15


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_prolongation_reproduces_polynomials(mg, orc, p):
    """On Cartesian cells a polynomial of degree p per variable lies in both spaces: prolonging its
    coarse nodal values gives its fine nodal values (fails for a transposed matrix, a swapped child
    bit or a wrong child cell)."""
    mc = synth.box_mesh(2, 1, 3)
    mf = synth.refine(mc)
    C = np.random.default_rng(p).uniform(-1, 1, (p + 1,) * 3)

    def f(X):
        return sum(C[a, b, c] * X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** c
                   for a in range(p + 1) for b in range(p + 1) for c in range(p + 1))

    uf = mg.prolong(mc, p, f(orc.node_coords(mc, p)))
    assert np.abs(uf - f(orc.node_coords(mf, p))).max() < 1e-12


@pytest.mark.parametrize("p", [1, 2, 3])
def test_transfer_lemmas(mg, orc, p):
    """Lemma prolongation_commutativity, P_cell G_c = G_f P_CG, and Lemma restriction_equivalence,
    G_c^T R_cell = P_CG^T G_f^T, on a curved mesh, with P_CG built from the global bases; and the
    duality <R r, G_c v> = <r, P G_c v>."""
    mc = synth.box_mesh(3, perturb=0.3)
    mf = synth.refine(mc)
    P = mg.prolongation_global(mc, p)
    u = synth.global_vector(mc, p, seed=1)
    lhs = mg.prolong(mc, p, orc.gather(mc, p, u))
    assert np.abs(lhs - orc.gather(mf, p, P @ u)).max() < 1e-13
    r = synth.cellwise_random(mf, p, seed=2)
    rc = mg.restrict(mc, p, r)
    ref = P.T @ orc.scatter_add(mf, p, r)
    assert np.abs(orc.scatter_add(mc, p, rc) - ref).max() < 1e-13 * np.abs(ref).max()
    v = orc.gather(mc, p, synth.global_vector(mc, p, seed=3))
    assert abs(rc @ v - r @ mg.prolong(mc, p, v)) < 1e-12 * np.abs(r).sum()


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("kind", [1, 2, 3], ids=["K", "M", "K+M"])
def test_galerkin_identity_on_cartesian_cells(mg, orc, p, kind):
    """Nested spaces with exact quadrature (Cartesian cells, p+1 Gauss points): the coarse operator
    is the Galerkin product P_CG^T A_f P_CG."""
    mc = synth.box_mesh(2, 1, 2)
    mf = synth.refine(mc)
    P = mg.prolongation_global(mc, p)
    Ac = orc.assemble_global(mc, p, kind).toarray()
    G = (P.T @ orc.assemble_global(mf, p, kind) @ P).toarray()
    assert np.abs(G - Ac).max() < 1e-12 * np.abs(Ac).max()


def three_levels(mg, p, kind=1, perturb=0.3):
    m0 = synth.box_mesh(3, perturb=perturb)
    m1 = synth.refine(m0)
    m2 = synth.refine(m1)
    return mg.hierarchy([m0, m1, m2], p, kind)


@pytest.mark.parametrize("p", [1, 2])
def test_smoother_forms_agree(mg, orc, p):
    """Lemma smoother_equivalence and Eq. (deferred_assembly): the literal cell-wise sweep, the
    fused sweep (valence-baked diagonal, averaging DSS at the end) and the gathered assembled damped
    Jacobi step u + omega D^-1 (b - A u) on the interior DoFs give the same iterate."""
    L = three_levels(mg, p)[1]
    m = L.mesh
    ug = synth.global_vector(m, p, seed=3)
    u = orc.gather(m, p, ug)
    b = synth.cellwise_random(m, p, seed=4)
    s1 = mg.smooth(L, b, u, 0.7)
    s2 = mg.smooth_fused(L, b, u, 0.7)
    s3 = orc.gather(m, p, ug + 0.7 * L.dinv_g * (orc.scatter_add(m, p, b) - L.A @ ug))
    scale = np.abs(s1).max()
    assert np.abs(s1 - s2).max() < 1e-14 * scale and np.abs(s1 - s3).max() < 1e-14 * scale


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("fused", [False, True], ids=["literal", "fused"])
def test_vcycle_equals_classical(mg, orc, p, fused):
    """Theorem mg_local_equivalence on a uniform hierarchy of curved meshes: one cell-wise V-cycle
    on (raw b, continuous u) is the gather of one classical V-cycle on (G^T b, u_CG)."""
    lv = three_levels(mg, p)
    m = lv[2].mesh
    ug = synth.global_vector(m, p, seed=5)
    b = synth.cellwise_random(m, p, seed=6)
    v1 = mg.vcycle(lv, 2, b, orc.gather(m, p, ug), fused=fused)
    v2 = orc.gather(m, p, mg.vcycle_assembled(lv, 2, orc.scatter_add(m, p, b), ug))
    assert np.abs(v1 - v2).max() < 1e-13 * np.abs(v2).max()


def test_coarse_grid_correction_is_a_galerkin_projection(mg, orc):
    """Without smoothing, one two-level cycle on Cartesian cells (A_c = P^T A_f P) leaves a residual
    whose restriction vanishes on the coarse interior DoFs."""
    p = 2
    lv = mg.hierarchy([synth.box_mesh(2, 3, 2), synth.refine(synth.box_mesh(2, 3, 2))], p, 1)
    m = lv[1].mesh
    b = synth.cellwise_random(m, p, seed=7)
    u0 = orc.gather(m, p, synth.global_vector(m, p, seed=8) * lv[1].mask)
    u1 = mg.vcycle(lv, 1, b, u0, nu1=0, nu2=0)
    rc = orc.scatter_add(lv[0].mesh, p, mg.restrict(lv[0].mesh, p, b - lv[1].apply(u1)))
    r0 = orc.scatter_add(lv[0].mesh, p, mg.restrict(lv[0].mesh, p, b - lv[1].apply(u0)))
    assert np.abs(lv[0].mask * rc).max() < 1e-12 * np.abs(lv[0].mask * r0).max()


@pytest.mark.parametrize("p,levels", [(1, (2, 3, 4)), (2, (2, 3, 4)), (3, (2, 3))])
def test_mg_pcg_solves_level_independently(mg, orc, p, levels):
    """The V-cycle-preconditioned CG on the Cartesian cube reaches 1e-10 in a handful of iterations
    that does not grow with the number of levels (the paper reports 8-11 on the cube for a 1e-14
    energy reduction), and its solution is the direct solve's."""
    its = []
    for nl in levels:
        ms = [synth.box_mesh(2)]
        for _ in range(nl - 1):
            ms.append(synth.refine(ms[-1]))
        lv = mg.hierarchy(ms, p, 1)
        b = orc.load_vector(ms[-1], p)
        u, k, res = mg.mg_pcg(lv, b, tol=1e-10)
        assert res <= 1e-10
        top = lv[-1]
        if top.mesh.ncells <= 512:  # the sparse direct solve is slow beyond 8^3 cells
            ud = orc.gather(top.mesh, p, orc.direct_solve(top.A, orc.scatter_add(top.mesh, p, b), top.mask))
            assert np.abs(u - ud).max() < 1e-8 * np.abs(ud).max()
        its.append(k)
    assert max(its) <= 12 and max(its) - min(its) <= 3, its


def cube_levels(mg, p, nl):
    ms = [synth.box_mesh(2)]
    for _ in range(nl - 1):
        ms.append(synth.refine(ms[-1]))
    return mg.hierarchy(ms, p, 1)


def test_energy_measure_is_the_error_pairing(mg, orc):
    """Eq. (energy_measure): eta(u) = <b - A u, u> = a(e, u) with e = u* - u, zero at the solution."""
    p = 2
    L = cube_levels(mg, p, 2)[1]
    m = L.mesh
    b = orc.load_vector(m, p)
    us = orc.direct_solve(L.A, orc.scatter_add(m, p, b), L.mask)
    ug = synth.global_vector(m, p, seed=9) * L.mask
    eta = mg.energy_measure(L, b, orc.gather(m, p, ug))
    assert abs(eta - (us - ug) @ (L.A @ ug)) < 1e-12 * abs(eta)
    assert abs(mg.energy_measure(L, b, orc.gather(m, p, us))) < 1e-12 * abs(eta)


@pytest.mark.parametrize("p,nl", [(1, 2), (1, 3), (2, 2), (2, 3), (3, 2), (3, 3)])
def test_vcycle_iteration_contracts(mg, orc, p, nl):
    """The V-cycle as a stationary iteration (the paper's fixed number of cycles) reduces the
    energy-norm error by a level-independent factor well below one (0.03-0.3 measured here)."""
    lv = cube_levels(mg, p, nl)
    L = lv[-1]
    m = L.mesh
    b = orc.load_vector(m, p)
    us = orc.direct_solve(L.A, orc.scatter_add(m, p, b), L.mask)
    kg = orc.scatter_add(m, p, np.ones_like(b))
    u = np.zeros_like(b)
    errs = []
    for _ in range(5):
        u = mg.vcycle(lv, nl - 1, b, u)
        e = us - orc.scatter_add(m, p, u) / kg
        errs.append(np.sqrt(e @ (L.A @ e)))
    ratios = np.array(errs[1:]) / np.array(errs[:-1])
    assert ratios.max() < 0.4, ratios


def test_vcycle_reads_its_input_only_through_the_assembly(mg, orc):
    """The cycle's output depends on the raw right-hand side only through G^T b: the averaged
    S-bar b gives the same correction (what lets a reduced-precision cycle take S-bar r)."""
    p = 2
    lv = three_levels(mg, p)
    L = lv[2]
    b = synth.cellwise_random(L.mesh, p, seed=10)
    z0 = mg.vcycle(lv, 2, b, np.zeros_like(b))
    z1 = mg.vcycle(lv, 2, mg.average(L, b), np.zeros_like(b))
    assert np.abs(z0 - z1).max() < 1e-13 * np.abs(z0).max()


@pytest.mark.parametrize("p,nl", [(2, 3), (3, 3), (4, 2)])
def test_fp32_vcycle_preconditioner(mg, orc, p, nl):
    """An FP32-storage V-cycle inside the FP64 CG, fed the averaged residual, converges like the
    FP64 cycle (same iterations within one, true assembled residual <= 1e-9); fed the raw residual
    instead, the rounding of the copies' partial integrals stalls the true residual near 1e-8."""
    lv = cube_levels(mg, p, nl)
    L = lv[-1]
    m = L.mesh
    b = orc.load_vector(m, p)

    def true_res(u):
        return (np.linalg.norm(L.mask * orc.scatter_add(m, p, b - L.apply(u)))
                / np.linalg.norm(L.mask * orc.scatter_add(m, p, b)))

    _, k64, _ = mg.mg_pcg(lv, b, tol=1e-10)
    u32, k32, _ = mg.mg_pcg(lv, b, tol=1e-10, dtype=np.float32)
    assert abs(k32 - k64) <= 1 and true_res(u32) <= 1e-9, (k64, k32, true_res(u32))
    raw = np.zeros_like(b)  # the same CG with the raw residual rounded into the cycle
    r = b.copy()
    z = mg.vcycle(lv, nl - 1, r, np.zeros_like(r), dtype=np.float32)
    d = z.copy()
    rho = r @ z
    for _ in range(k64):
        q = L.apply(d)
        a = rho / (d @ q)
        raw, r = raw + a * d, r - a * q
        z = mg.vcycle(lv, nl - 1, r, np.zeros_like(r), dtype=np.float32)
        rho, rho_old = r @ z, rho
        d = z + (rho / rho_old) * d
    assert true_res(raw) > 1e-9
