"""Pins for the oracle's global numbering, G, G^T, S (Sec. 2.1; Sec. 4.1 Eq. (dss_operator);
Sec. 5 Eq. (averaging_dss)), the assembled matrix (Eq. (constrained_system)) and the diagonal
(Eq. (jacobi_recap))."""
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def valence_closed_form(mesh, p):
    """Number of cells sharing each global DoF: per axis 2 on interior cell-boundary planes, else 1."""
    def axis(nc):
        g = np.arange(nc * p + 1)
        return np.where((g % p == 0) & (g > 0) & (g < nc * p), 2, 1)
    kz, ky, kx = np.meshgrid(axis(mesh.nz), axis(mesh.ny), axis(mesh.nx), indexing="ij")
    return (kx * ky * kz).ravel().astype(float)


@pytest.mark.parametrize("p", [1, 2, 5])
def test_valence(orc, p):
    mesh = synth.box_mesh(3, 2, 4)
    kappa = orc.scatter_add(mesh, p, np.ones(mesh.ncells * (p + 1) ** 3))
    assert np.array_equal(kappa, valence_closed_form(mesh, p))


@pytest.mark.parametrize("p", [1, 3])
def test_dss_identities(orc, p):
    mesh = synth.box_mesh(3, 4, 2)
    kappa = valence_closed_form(mesh, p)
    u = synth.global_vector(mesh, p, seed=4)
    r = synth.cellwise_random(mesh, p, seed=5)
    Gu = orc.gather(mesh, p, u)
    # S G u = G (kappa u): each copy receives the sum of all kappa identical copies
    assert np.allclose(orc.dss(mesh, p, Gu), orc.gather(mesh, p, kappa * u), atol=1e-14, rtol=0)
    # <S r, r> = ||G^T r||^2
    Sr = orc.dss(mesh, p, r)
    GTr = orc.scatter_add(mesh, p, r)
    assert abs(Sr @ r - GTr @ GTr) < 1e-12 * (GTr @ GTr)
    # Im S in Im G: S r is continuous (copies agree), and S is symmetric
    gmap = orc.global_index(mesh, p)
    first = np.full(len(kappa), np.nan)
    first[gmap[::-1]] = Sr[::-1]
    assert np.allclose(Sr, first[gmap], atol=1e-14, rtol=0)
    r2 = synth.cellwise_random(mesh, p, seed=6)
    assert abs(orc.dss(mesh, p, r2) @ r - Sr @ r2) < 1e-12
    # averaging DSS S_bar = G kappa^-1 G^T is a projection that fixes continuous vectors
    Sbar = lambda v: orc.gather(mesh, p, orc.scatter_add(mesh, p, v) / kappa)
    assert np.allclose(Sbar(Sbar(r)), Sbar(r), atol=1e-14)
    assert np.allclose(Sbar(Gu), Gu, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_valence_and_scaling_identities(orc, p):
    """Eq. (jacobi_recap): G D_CG^-1 = D_cell^-1 G (scaling intertwines with the gather), and
    Eq. (valence_baking): S_bar K_cell D_cell^-1 = D_cell^-1 S on raw vectors."""
    mesh = synth.box_mesh(3, 2, 3, perturb=0.2)
    d = orc.diagonal(mesh, p, 1)
    u = synth.global_vector(mesh, p, seed=11)
    dinv_cell = orc.gather(mesh, p, 1.0 / d)
    assert np.array_equal(orc.gather(mesh, p, (1.0 / d) * u), dinv_cell * orc.gather(mesh, p, u))
    kcell = orc.gather(mesh, p, valence_closed_form(mesh, p))
    r = synth.cellwise_random(mesh, p, seed=12)
    kappa_g = orc.scatter_add(mesh, p, np.ones_like(r))
    lhs = orc.gather(mesh, p, orc.scatter_add(mesh, p, kcell * dinv_cell * r) / kappa_g)
    rhs = dinv_cell * orc.dss(mesh, p, r)
    assert np.abs(lhs - rhs).max() < 1e-14 * np.abs(rhs).max()


def test_pairing_identity(orc):
    """<f~, G u> = <G^T f~, u> (Sec. 2.1, Eq. (pairing_global))."""
    mesh = synth.box_mesh(2, 3, 3, perturb=0.2)
    p = 3
    f = synth.cellwise_random(mesh, p, seed=7)
    u = synth.global_vector(mesh, p, seed=8)
    assert abs(f @ orc.gather(mesh, p, u) - orc.scatter_add(mesh, p, f) @ u) < 1e-12


def test_q1_assembled_stencil(orc):
    coef = {}
    for line in open(os.path.join(GOLDEN, "q1_stencil.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        coef[k] = float(v)
    N = 4
    mesh = synth.box_mesh(N)
    A = orc.assemble_global(mesh, 1, orc.KIND_LAPLACE).toarray()
    h = 1.0 / N
    gx = N + 1
    c = 2 + gx * (2 + gx * 2)  # interior vertex (2,2,2)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                nnz = abs(dx) + abs(dy) + abs(dz)
                key = ["centre", "face", "edge", "corner"][nnz]
                assert abs(A[c, c + dx + gx * (dy + gx * dz)] - h * coef[key]) < 1e-14


@pytest.mark.parametrize("p,kind", [(1, 1), (2, 3), (4, 2)])
def test_assembly_and_diagonal(orc, p, kind):
    """A_CG = G^T A G: (G^T A G) u_g from the cell-wise apply equals the sparse global matrix times
    u_g, and the oracle diagonal equals diag(A_CG)."""
    mesh = synth.box_mesh(2, 3, 2, perturb=0.2)
    A = orc.assemble_global(mesh, p, kind)
    u = synth.global_vector(mesh, p, seed=9)
    lhs = orc.scatter_add(mesh, p, orc.apply_local(mesh, p, kind, orc.gather(mesh, p, u)))
    assert np.abs(lhs - A @ u).max() < 1e-12 * np.abs(A @ u).max()
    assert np.abs(orc.diagonal(mesh, p, kind) - A.diagonal()).max() < 1e-13 * A.diagonal().max()
    assert abs(A - A.T).max() < 1e-14 * abs(A).max()
