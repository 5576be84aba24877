"""Geometric multigrid of a uniform mesh hierarchy in cell-wise storage, FP64 (Sec. 3-5).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: the CUDA library never imports or calls it.

Levels: level 0 is a box mesh, level l+1 splits every cell of level l into 2 x 2 x 2 children by
the cell's own trilinear map (the input generator's ``refine``), so the spaces V_0 c V_1 c ... are
nested (Sec. 3). Cells are numbered lexicographically on every level; child c = bx + 2 by + 4 bz of
coarse cell (cx, cy, cz) is fine cell (2cx+bx, 2cy+by, 2cz+bz).

What is here, each following the paper's steps in its order:
  * the cell-wise transfers (Algorithms prolongation and restriction; the loops are in oracle.c);
  * the classical prolongation P_CG between the global spaces, built a second way (from the global
    nodal bases in the hierarchy's logical coordinates) for the equivalence pins of Sec. 3;
  * the cell-wise damped Jacobi smoother, literally (Eq. (cellwise_smoother), Algorithm smoother)
    and in the fused form the paper executes (Eq. (deferred_assembly), Algorithm smoother_fused);
  * the V-cycle (Algorithm mg_vcycle) on cell-wise vectors, beside the classical V-cycle on the
    assembled system it is equivalent to;
  * CG preconditioned by one V-cycle from a zero initial guess, in the cell-wise primal-dual form.

Readings where the paper is silent (also listed with the design notes):
  * coarse solve A_0^{-1}: sparse direct solve of the assembled level-0 system on its interior DoFs,
    gathered back to cells;
  * nu1 = nu2 = 2 smoothing sweeps and omega = 0.7 by default (the paper's cube settings);
  * homogeneous Dirichlet on the cube boundary on every level, by zeros of the inverse diagonal
    (Sec. 5, constraints baked into the diagonal); a uniform hierarchy has no refinement edge, so
    the masks of the local smoother are the identity;
  * the preconditioned CG stops when sqrt(<r, z> / <r_0, z_0>) <= tol.
"""
import numpy as np

from . import (_dp, apply_local, assemble_global, boundary_mask_global, diagonal, direct_solve, dss, gather,
               gll, lagrange, lib, scatter_add)


# --------------------------------------------------------------- transfers
def prolongation_1d(p):
    """(P_0, P_1): P_b[i][a] = l_a((xi_i + b) / 2), the parent's basis at the nodes of child b."""
    n = p + 1
    P0, P1 = np.zeros((n, n)), np.zeros((n, n))
    lib().orc_prolong_1d(p, _dp(P0), _dp(P1))
    return P0, P1


def prolong(mesh_c, p, uc):
    """Algorithm prolongation: coarse cell-wise primal -> fine cell-wise primal (8x the cells)."""
    uc = np.ascontiguousarray(uc, dtype=np.float64)
    uf = np.zeros(8 * uc.size)
    lib().orc_prolong(mesh_c.nx, mesh_c.ny, mesh_c.nz, p, _dp(uc), _dp(uf))
    return uf


def restrict(mesh_c, p, rf):
    """Algorithm restriction: fine raw (unassembled) dual -> coarse raw dual, additive over children."""
    rf = np.ascontiguousarray(rf, dtype=np.float64)
    rc = np.zeros(rf.size // 8)
    lib().orc_restrict(mesh_c.nx, mesh_c.ny, mesh_c.nz, p, _dp(rf), _dp(rc))
    return rc


def prolongation_global(mesh_c, p):
    """Classical prolongation P_CG: V_CG,l-1 -> V_CG,l (sparse, global numbering of both levels).

    Built from the global nodal bases, not from the cell loops: along each axis the coarse space is
    the piecewise Q_p space on the logical coarse grid, so entry (f, g) of the 1D factor is coarse
    global basis function g evaluated at the logical coordinate of fine global node f; the 3D
    matrix is the Kronecker product of the three factors (x fastest)."""
    import scipy.sparse as sp
    xi = gll(p)

    def axis(nc):
        gc, gf = nc * p + 1, 2 * nc * p + 1
        M = np.zeros((gf, gc))
        for f in range(gf):
            cf = min(f // p, 2 * nc - 1)       # fine cell holding node f, and its local index
            t = (cf + xi[f - cf * p]) / 2.0     # the node in coarse-cell units
            cc = min(int(np.floor(t)), nc - 1)
            l, _ = lagrange(xi, t - cc)
            M[f, cc * p: cc * p + p + 1] = l
        return sp.csr_matrix(M)

    return sp.kron(axis(mesh_c.nz), sp.kron(axis(mesh_c.ny), axis(mesh_c.nx))).tocsr()


# ------------------------------------------------------------------ levels
class Level:
    """One level: mesh, operator kind and the data the smoother and the coarse solve read."""

    def __init__(self, mesh, p, kind, coarse_mesh=None):
        self.mesh, self.p, self.kind = mesh, p, kind
        self.coarse_mesh = coarse_mesh
        self.mask = boundary_mask_global(mesh, p)                  # 0 on Dirichlet DoFs
        d = diagonal(mesh, p, kind)                                 # d = diag(A_CG)
        self.dinv_g = np.where(self.mask > 0, 1.0 / d, 0.0)
        self.dinv = gather(mesh, p, self.dinv_g)                    # D_cell^-1, Dirichlet zeros
        self.kappa = dss(mesh, p, np.ones(mesh.ncells * (p + 1) ** 3))  # valence of every copy
        self.dhat = self.kappa * self.dinv                          # K_cell D_cell^-1 (valence baked)
        self._A = None
        self._P = None

    @property
    def A(self):
        """Assembled A_CG of the level (coarse solve and the classical route)."""
        if self._A is None:
            self._A = assemble_global(self.mesh, self.p, self.kind)
        return self._A

    @property
    def P(self):
        """Classical prolongation from the level below into this one."""
        if self._P is None:
            self._P = prolongation_global(self.coarse_mesh, self.p)
        return self._P

    def apply(self, u):
        return apply_local(self.mesh, self.p, self.kind, u)


def hierarchy(meshes, p, kind):
    """Levels 0..L from the meshes of a uniform hierarchy (meshes[l+1] refines meshes[l])."""
    return [Level(m, p, kind, meshes[i - 1] if i else None) for i, m in enumerate(meshes)]


# ---------------------------------------------------------------- smoother
def smooth(level, b, u, omega):
    """Algorithm smoother, step by step: v = A u; r = b - v; dual mask (identity: no refinement
    edge); z = S r; c = omega D_cell^-1 z; u + c."""
    v = level.apply(u)
    r = b - v
    z = dss(level.mesh, level.p, r)
    return u + omega * level.dinv * z


def average(level, w):
    """S-bar w = G (G^T G)^-1 G^T w (Eq. (averaging_dss)): assemble, divide by the valence, re-inject."""
    return dss(level.mesh, level.p, w) / level.kappa


def smooth_fused(level, b, u, omega):
    """Algorithm smoother_fused: v = A u; u + omega D-hat^-1 (b - v) per copy; then S-bar."""
    v = level.apply(u)
    w = u + omega * level.dhat * (b - v)
    return average(level, w)


# ----------------------------------------------------------------- V-cycle
def coarse_solve(level, b):
    """u_0 = A_0^-1 b_0 on the interior DoFs of level 0, gathered to cells."""
    ug = direct_solve(level.A, scatter_add(level.mesh, level.p, b), level.mask)
    return gather(level.mesh, level.p, ug)


def stored(x, dtype):
    """x as held in memory of the given precision (FP64: unchanged; FP32: rounded to nearest)."""
    return x if dtype == np.float64 else x.astype(dtype).astype(np.float64)


def vcycle(levels, l, b, u, nu1=2, nu2=2, omega=0.7, fused=False, dtype=np.float64):
    """Algorithm mg_vcycle on cell-wise vectors: b raw dual, u continuous primal; returns u.
    ``dtype`` is the storage precision of every vector of the cycle (FP32 for the mixed-precision
    cycle: each step's result is rounded to it; the arithmetic of a step stays FP64)."""
    L = levels[l]
    b = stored(b, dtype)
    if l == 0:
        return stored(coarse_solve(L, b), dtype)
    sm = smooth_fused if fused else smooth
    u = stored(u, dtype)
    for _ in range(nu1):
        u = stored(sm(L, b, u, omega), dtype)
    r = stored(b - L.apply(u), dtype)
    bc = stored(restrict(levels[l - 1].mesh, L.p, r), dtype)
    e = vcycle(levels, l - 1, bc, np.zeros_like(bc), nu1, nu2, omega, fused, dtype)
    u = stored(u + prolong(levels[l - 1].mesh, L.p, e), dtype)
    for _ in range(nu2):
        u = stored(sm(L, b, u, omega), dtype)
    return u


def vcycle_assembled(levels, l, b, u, nu1=2, nu2=2, omega=0.7):
    """The classical V-cycle on the assembled systems (global vectors): damped Jacobi on the
    interior DoFs, restriction P_CG^T, prolongation P_CG, direct coarse solve."""
    L = levels[l]
    if l == 0:
        return direct_solve(L.A, b, L.mask)
    for _ in range(nu1):
        u = u + omega * L.dinv_g * (b - L.A @ u)
    r = b - L.A @ u
    e = vcycle_assembled(levels, l - 1, L.P.T @ r, np.zeros(L.P.shape[1]), nu1, nu2, omega)
    u = u + L.P @ e
    for _ in range(nu2):
        u = u + omega * L.dinv_g * (b - L.A @ u)
    return u


# ------------------------------------------------------------------ MG-PCG
def energy_measure(level, b, u):
    """eta(u) = <b - A u, u> (Eq. (energy_measure)): raw residual paired with the continuous iterate."""
    return float((b - level.apply(u)) @ u)


def mg_pcg(levels, b, tol=1e-10, maxit=200, nu1=2, nu2=2, omega=0.7, fused=False, dtype=np.float64):
    """CG on the finest level, cell-wise primal-dual form (residual raw, iterate and direction
    continuous), preconditioned by one V-cycle from a zero initial guess (Sec. 5: the cycle then
    starts from the residual itself). The CG runs in FP64; ``dtype`` is the storage precision of
    the V-cycle (FP32: the mixed-precision preconditioner the paper names as the next gain, Sec. 8).
    A reduced-precision cycle is fed the averaged residual S-bar r (Eq. (averaging_dss)): the raw
    residual's copies are O(1) partial integrals whose sum is tiny, and rounding them would destroy
    the assembled residual; the average has the same assembly (the cycle reads its input only
    through G^T) with every copy small. Returns (u, iterations, sqrt(<r,z>/<r_0,z_0>))."""
    top = len(levels) - 1
    L = levels[top]

    def precond(r):
        if dtype != np.float64:
            r = average(L, r)
        return vcycle(levels, top, r, np.zeros_like(r), nu1, nu2, omega, fused, dtype)

    u = np.zeros_like(b)
    r = b.copy()
    z = precond(r)
    d = z.copy()
    rho = r @ z
    rho0 = rho
    k = 0
    while k < maxit and np.sqrt(rho / rho0) > tol:
        q = L.apply(d)
        alpha = rho / (d @ q)
        u = u + alpha * d
        r = r - alpha * q
        z = precond(r)
        rho_new = r @ z
        d = z + (rho_new / rho) * d
        rho = rho_new
        k += 1
    return u, k, float(np.sqrt(rho / rho0))
