"""Pins for the oracle's solve chain: load vector, assembled Jacobi-PCG, error norms
(Poisson problem of Sec. 2, Eq. (poisson), homogeneous Dirichlet)."""
import numpy as np
import pytest

import synth


def solve(orc, mesh, p, which, tol=1e-12):
    A = orc.assemble_global(mesh, p, orc.KIND_LAPLACE)
    b = orc.scatter_add(mesh, p, orc.load_vector(mesh, p, which))
    mask = orc.boundary_mask_global(mesh, p)
    u, its, res, _ = orc.pcg_assembled(A, b, mask, tol=tol, maxit=5000)
    return A, b, mask, u, its, res


@pytest.mark.parametrize("p", [2, 3])
def test_bubble_solution_is_exact(orc, p):
    """u = x(1-x)y(1-y)z(1-z) lies in Q_p for p >= 2, so the Galerkin solution on an affine mesh is
    its interpolant (f is integrated exactly by p+1 Gauss points)."""
    mesh = synth.box_mesh(3, 2, 4)
    A, b, mask, u, its, res = solve(orc, mesh, p, orc.PROBLEM_BUBBLE)
    xyz = orc.node_coords(mesh, p)
    ucell = orc.gather(mesh, p, u)
    bub = np.prod(xyz * (1 - xyz), axis=1)
    assert np.abs(ucell - bub).max() < 1e-11
    l2, h1 = orc.error_norms(mesh, p, ucell, orc.PROBLEM_BUBBLE)
    assert l2 < 1e-11 and h1 < 1e-10


def test_pcg_matches_direct(orc):
    mesh = synth.box_mesh(3, 3, 3, perturb=0.2)
    p = 2
    A, b, mask, u, its, res = solve(orc, mesh, p, orc.PROBLEM_SINE, tol=1e-13)
    ud = orc.direct_solve(A, b, mask)
    assert res <= 1e-13
    assert np.abs(u - ud).max() < 1e-10 * np.abs(ud).max()


@pytest.mark.parametrize("p,perturb", [(1, 0.0), (2, 0.0), (2, 0.1), (3, 0.1)])
def test_convergence_orders(orc, p, perturb):
    """Optimal orders for the sine solution: L2 error O(h^(p+1)), H1 error O(h^p)."""
    Ns = [2, 4, 8] if p < 3 else [2, 4, 6]
    errs = []
    for N in Ns:
        mesh = synth.box_mesh(N, perturb=perturb)
        A, b, mask, u, its, res = solve(orc, mesh, p, orc.PROBLEM_SINE)
        errs.append(orc.error_norms(mesh, p, orc.gather(mesh, p, u)))
    e = np.array(errs)
    hs = 1.0 / np.array(Ns)
    rl2 = np.log(e[-2, 0] / e[-1, 0]) / np.log(hs[-2] / hs[-1])
    rh1 = np.log(e[-2, 1] / e[-1, 1]) / np.log(hs[-2] / hs[-1])
    assert rl2 > p + 1 - 0.3, (rl2, e)
    assert rh1 > p - 0.25, (rh1, e)
