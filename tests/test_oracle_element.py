"""Pins for the oracle's element matrices and cell-local operator (Sec. 2, Eq. (poisson);
Sec. 2.1, the cell-local operator A; Sec. 6, the factored Cartesian operator)."""
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def unit_cube_vertices(h=1.0, origin=(0, 0, 0)):
    return np.array([[origin[0] + a * h, origin[1] + b * h, origin[2] + c * h]
                     for c in (0, 1) for b in (0, 1) for a in (0, 1)], float)


def test_q1_unit_cube_closed_form(orc):
    rows = {}
    for line in open(os.path.join(GOLDEN, "q1_unit_cube.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, *vals = line.split()
        rows[name] = np.array([float(v) for v in vals])
    K, M = orc.element_matrices(1, unit_cube_vertices())
    assert np.allclose(K[0] * 12, rows["K_row0_times_12"], atol=1e-13)
    assert np.allclose(M[0] * 216, rows["M_row0_times_216"], atol=1e-13)


def one_d_matrices(p):
    """1D stiffness / mass matrices of the GLL Lagrange basis on [0,1], built independently of the
    oracle in 30-digit arithmetic: nodes as roots of P_p' (mpmath.polyroots), basis by the product
    formula, integrals by mpmath.quad."""
    import mpmath as mp
    mp.mp.dps = 30
    # coefficients of P_p' in the monomial basis, highest degree first
    Pp = mp.taylor(lambda t: mp.legendre(p, t), 0, p)        # P_p(t) = sum c_k t^k
    dcoef = [k * Pp[k] for k in range(p, 0, -1)]              # P_p'(t), highest first
    roots = sorted(mp.re(r) for r in mp.polyroots(dcoef, maxsteps=200, extraprec=60)) if p > 1 else []
    nodes = [mp.mpf(0)] + [(1 + r) / 2 for r in roots] + [mp.mpf(1)]
    n = p + 1

    def ell(i, x):
        v = mp.mpf(1)
        for m in range(n):
            if m != i:
                v *= (x - nodes[m]) / (nodes[i] - nodes[m])
        return v

    def dell(i, x):
        return mp.diff(lambda t: ell(i, t), x)
    K1 = np.zeros((n, n))
    M1 = np.zeros((n, n))
    for i in range(n):
        for j in range(i, n):
            K1[i, j] = K1[j, i] = float(mp.quad(lambda x: dell(i, x) * dell(j, x), [0, 1]))
            M1[i, j] = M1[j, i] = float(mp.quad(lambda x: ell(i, x) * ell(j, x), [0, 1]))
    return K1, M1


@pytest.mark.parametrize("p", range(1, 8))
def test_factored_cartesian_form(orc, p):
    """On an h-cube the element matrices are h(K1(x)M1(x)M1 + ...) and h^3 M1(x)M1(x)M1, the
    factored tensor-product form with the per-element scalar det J J^-2 = h (Sec. 6)."""
    h = 0.125
    K, M = orc.element_matrices(p, unit_cube_vertices(h, (0.25, 0.5, 0.125)))
    K1, M1 = one_d_matrices(p)
    # local index i + n(j + n k): numpy kron order (z, y, x)
    Kf = h * (np.kron(M1, np.kron(M1, K1)) + np.kron(M1, np.kron(K1, M1)) + np.kron(K1, np.kron(M1, M1)))
    Mf = h ** 3 * np.kron(M1, np.kron(M1, M1))
    assert np.abs(K - Kf).max() <= 1e-12 * np.abs(Kf).max()
    assert np.abs(M - Mf).max() <= 1e-12 * np.abs(Mf).max()


@pytest.mark.parametrize("p", range(1, 8))
def test_curved_cell_invariants(orc, p):
    mesh = synth.box_mesh(3, 3, 3, perturb=0.3)
    X = orc.cell_vertices(mesh, 13)  # the centre cell, all vertices displaced
    K, M = orc.element_matrices(p, X)
    n3 = (p + 1) ** 3
    assert np.abs(K - K.T).max() < 1e-14 * np.abs(K).max()
    assert np.abs(K @ np.ones(n3)).max() < 1e-12 * np.abs(K).max()          # Laplace kills constants
    assert np.linalg.eigvalsh(M).min() > 0                                     # mass is SPD
    ev = np.linalg.eigvalsh(K)
    assert ev.min() > -1e-12 * ev.max() and np.sum(ev < 1e-10 * ev.max()) == 1  # one-dim. kernel


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_physical_coordinate_functions_curved(orc, p):
    """x, y, z are in the trilinear-mapped space, so with I(x) the interpolant of the physical
    x-coordinate, I(x)^T K I(x) = |Omega| and I(x)^T K I(y) = 0 on curved meshes (grad x = e_x at
    every quadrature point), and 1^T M 1 = |Omega| = 1 (detJ integrated exactly)."""
    mesh = synth.box_mesh(3, 2, 2, perturb=0.25)
    xyz = orc.node_coords(mesh, p)
    one = np.ones(len(xyz))
    Kx = orc.apply_local(mesh, p, orc.KIND_LAPLACE, xyz[:, 0])
    assert abs(xyz[:, 0] @ Kx - 1.0) < 1e-12
    assert abs(xyz[:, 1] @ Kx) < 1e-12
    Ky = orc.apply_local(mesh, p, orc.KIND_LAPLACE, xyz[:, 1])
    assert abs(xyz[:, 2] @ Ky) < 1e-12
    assert abs(one @ orc.apply_local(mesh, p, orc.KIND_MASS, one) - 1.0) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_mass_integrates_polynomials_curved(orc, p):
    """1^T M I(x^a y^b z^c) = 1/((a+1)(b+1)(c+1)) for a+b+c <= p on the curved unit cube."""
    mesh = synth.box_mesh(3, 3, 2, perturb=0.3)
    xyz = orc.node_coords(mesh, p)
    one = np.ones(len(xyz))
    M1 = orc.apply_local(mesh, p, orc.KIND_MASS, one)
    for a in range(p + 1):
        for b in range(p + 1 - a):
            c = p - a - b
            u = xyz[:, 0] ** a * xyz[:, 1] ** b * xyz[:, 2] ** c
            assert abs(M1 @ u - 1.0 / ((a + 1) * (b + 1) * (c + 1))) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_stiffness_integrates_polynomials_affine(orc, p):
    """I(u)^T K I(v) = int grad u . grad v for u, v in Q_p on an affine mesh."""
    mesh = synth.box_mesh(2, 3, 2)
    xyz = orc.node_coords(mesh, p)
    x, y, z = xyz.T
    a, b = min(p, 2), min(p, 1)
    u = x ** a * y ** b               # grad u = (a x^(a-1) y^b, b x^a y^(b-1), 0)
    v = x ** b * z ** a               # grad v = (b x^(b-1) z^a, 0, a x^b z^(a-1))
    Kv = orc.apply_local(mesh, p, orc.KIND_LAPLACE, v)
    # only the x-components meet: int a b x^(a+b-2) y^b z^a
    exact = (a * b / (a + b - 1) / (b + 1) / (a + 1)) if a + b > 1 else (a * b / (b + 1) / (a + 1))
    assert abs(u @ Kv - exact) < 1e-12


@pytest.mark.parametrize("p", [1, 3, 6])
def test_symmetry_continuous(orc, p):
    mesh = synth.box_mesh(2, 2, 3, perturb=0.2)
    x = orc.gather(mesh, p, synth.global_vector(mesh, p, seed=1))
    y = orc.gather(mesh, p, synth.global_vector(mesh, p, seed=2))
    for kind in (1, 2, 3):
        Ay = orc.apply_local(mesh, p, kind, y)
        Ax = orc.apply_local(mesh, p, kind, x)
        assert abs(x @ Ay - y @ Ax) < 1e-12 * abs(x @ Ay)


def test_apply_cell_subset_matches_full(orc):
    mesh = synth.box_mesh(3, 2, 2, perturb=0.2)
    p = 2
    x = synth.cellwise_random(mesh, p, seed=3)
    full = orc.apply_local(mesh, p, 3, x).reshape(mesh.ncells, -1)
    cells = np.array([5, 0, 11])
    assert np.array_equal(orc.apply_local(mesh, p, 3, x, cells), full[cells])
