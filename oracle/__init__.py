"""Plain FP64 CPU oracle for the cell-wise FEM hot path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py``. The CUDA library never imports, links or calls anything here.

Pieces:
  * ``oracle.c`` (compiled to ``_build/liboracle.so`` with gcc -O2 -fopenmp): 1D Gauss and
    Gauss-Lobatto rules, explicit element matrices, the cell-local apply, global numbering, G, G^T,
    S = G G^T, the assembled diagonal, the load vector and error norms;
  * this module: ctypes wrappers, the global sparse matrix A_CG = G^T A G assembled by
    brute force (Sec. 2.1, Eq. (constrained_system)), and an assembled Jacobi-preconditioned CG on
    the interior DoFs (homogeneous Dirichlet), plus a sparse direct solve;
  * ``oracle.mg``: the geometric multigrid of a uniform mesh hierarchy (Sec. 3 and 5): cell-wise
    transfers, the cell-wise damped Jacobi smoother in its literal and fused forms, the V-cycle and
    the V-cycle-preconditioned CG, beside the classical assembled V-cycle they are equivalent to;
  * ``oracle.dist``: the DSS and the Jacobi-PCG of a mesh split into z-slabs over torch.distributed
    ranks (face-layer exchange per slab interface, sums over ranks for the inner products);
  * ``oracle.mblock``: multi-block meshes (structured blocks glued face to face in any orientation):
    the global numbering by node position, G, G^T, S and the assembled A_CG across block interfaces.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

KIND_LAPLACE, KIND_MASS, KIND_LAPLACE_MASS = 1, 2, 3


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (plain gcc, no arch-specific flags)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.POINTER
        d, i64, c_int = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        dp, lp = P(d), P(i64)
        L.orc_gauss.argtypes = [c_int, dp, dp]
        L.orc_gll.argtypes = [c_int, dp]
        L.orc_lagrange.argtypes = [c_int, dp, d, dp, dp]
        L.orc_element_matrices.argtypes = [c_int, dp, dp, dp]
        L.orc_cell_vertices.argtypes = [c_int, c_int, c_int, dp, i64, dp]
        L.orc_apply_local.argtypes = [c_int, c_int, c_int, dp, c_int, c_int, dp, dp, i64, lp]
        L.orc_apply_local.restype = i64
        L.orc_global_index.argtypes = [c_int, c_int, c_int, c_int, lp]
        L.orc_gather.argtypes = [c_int, c_int, c_int, c_int, dp, dp]
        L.orc_scatter_add.argtypes = [c_int, c_int, c_int, c_int, dp, dp]
        L.orc_dss.argtypes = [c_int, c_int, c_int, c_int, dp, dp]
        L.orc_diagonal.argtypes = [c_int, c_int, c_int, dp, c_int, c_int, dp]
        L.orc_all_element_matrices.argtypes = [c_int, c_int, c_int, dp, c_int, c_int, dp]
        L.orc_all_element_matrices.restype = i64
        L.orc_load_vector.argtypes = [c_int, c_int, c_int, dp, c_int, c_int, dp]
        L.orc_error_norms.argtypes = [c_int, c_int, c_int, dp, c_int, c_int, c_int, dp, dp]
        L.orc_node_coords.argtypes = [c_int, c_int, c_int, dp, c_int, dp]
        L.orc_prolong_1d.argtypes = [c_int, dp, dp]
        L.orc_prolong.argtypes = [c_int, c_int, c_int, c_int, dp, dp]
        L.orc_restrict.argtypes = [c_int, c_int, c_int, c_int, dp, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------------ 1D rules
def gauss(q):
    x, w = np.zeros(q), np.zeros(q)
    assert lib().orc_gauss(q, _dp(x), _dp(w)) == 0
    return x, w


def gll(p):
    x = np.zeros(p + 1)
    assert lib().orc_gll(p, _dp(x)) == 0
    return x


def lagrange(nodes, xi):
    nodes = _f64(nodes)
    n = len(nodes)
    l, dl = np.zeros(n), np.zeros(n)
    lib().orc_lagrange(n, _dp(nodes), float(xi), _dp(l), _dp(dl))
    return l, dl


# ------------------------------------------------------------ element level
def element_matrices(p, X):
    """K, M (n^3 x n^3) of one cell with vertices X[8][3] (vertex a + 2b + 4c at (a,b,c))."""
    n3 = (p + 1) ** 3
    X = _f64(X).reshape(8, 3)
    K, M = np.zeros((n3, n3)), np.zeros((n3, n3))
    rc = lib().orc_element_matrices(p, _dp(X), _dp(K), _dp(M))
    if rc != 0:
        raise ValueError("non-positive Jacobian determinant")
    return K, M


def cell_vertices(mesh, e):
    X = np.zeros((8, 3))
    lib().orc_cell_vertices(mesh.nx, mesh.ny, mesh.nz, _dp(mesh.verts), int(e), _dp(X))
    return X


# --------------------------------------------------------------- mesh level
def apply_local(mesh, p, kind, x, cells=None):
    """y = A x cell by cell (LOCAL, unassembled dual). With ``cells`` only those cells of y are
    computed and returned as an array [len(cells)][n^3]."""
    x = _f64(x)
    n3 = (p + 1) ** 3
    y = np.zeros_like(x)
    if cells is None:
        bad = lib().orc_apply_local(mesh.nx, mesh.ny, mesh.nz, _dp(mesh.verts), p, kind, _dp(x),
                                    _dp(y), 0, None)
        if bad:
            raise ValueError(f"{bad} cells with non-positive Jacobian")
        return y
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    bad = lib().orc_apply_local(mesh.nx, mesh.ny, mesh.nz, _dp(mesh.verts), p, kind, _dp(x), _dp(y),
                                len(cells), _lp(cells))
    if bad:
        raise ValueError(f"{bad} cells with non-positive Jacobian")
    return y.reshape(-1, n3)[cells].copy()


def global_index(mesh, p):
    L = mesh.ncells * (p + 1) ** 3
    m = np.zeros(L, dtype=np.int64)
    lib().orc_global_index(mesh.nx, mesh.ny, mesh.nz, p, _lp(m))
    return m


def global_len(mesh, p):
    return (mesh.nx * p + 1) * (mesh.ny * p + 1) * (mesh.nz * p + 1)


def gather(mesh, p, ug):
    ug = _f64(ug)
    xc = np.zeros(mesh.ncells * (p + 1) ** 3)
    lib().orc_gather(mesh.nx, mesh.ny, mesh.nz, p, _dp(ug), _dp(xc))
    return xc


def scatter_add(mesh, p, yc):
    yc = _f64(yc)
    fg = np.zeros(global_len(mesh, p))
    lib().orc_scatter_add(mesh.nx, mesh.ny, mesh.nz, p, _dp(yc), _dp(fg))
    return fg


def dss(mesh, p, yc):
    """S y = G G^T y (Sec. 4.1, Eq. (dss_operator))."""
    yc = _f64(yc)
    z = np.zeros_like(yc)
    lib().orc_dss(mesh.nx, mesh.ny, mesh.nz, p, _dp(yc), _dp(z))
    return z


def diagonal(mesh, p, kind):
    """Assembled diagonal d = G^T diag(A_K) (global vector)."""
    d = np.zeros(global_len(mesh, p))
    lib().orc_diagonal(mesh.nx, mesh.ny, mesh.nz, _dp(mesh.verts), p, kind, _dp(d))
    return d


def all_element_matrices(mesh, p, kind):
    n3 = (p + 1) ** 3
    A = np.zeros((mesh.ncells, n3, n3))
    bad = lib().orc_all_element_matrices(mesh.nx, mesh.ny, mesh.nz, _dp(mesh.verts), p, kind, _dp(A))
    if bad:
        raise ValueError("non-positive Jacobian")
    return A


PROBLEM_SINE, PROBLEM_BUBBLE = 0, 1


def load_vector(mesh, p, which=PROBLEM_SINE):
    """Unassembled dual b_K,i = int_K f phi_i (q = p+1 Gauss points) for the manufactured problem
    ``which``: PROBLEM_SINE (u = sin(pi x) sin(pi y) sin(pi z), f = 3 pi^2 u) or PROBLEM_BUBBLE
    (u = x(1-x)y(1-y)z(1-z))."""
    b = np.zeros(mesh.ncells * (p + 1) ** 3)
    lib().orc_load_vector(mesh.nx, mesh.ny, mesh.nz, _dp(mesh.verts), p, which, _dp(b))
    return b


def error_norms(mesh, p, u_cell, which=PROBLEM_SINE, nq=None):
    """(L2 error, H1-seminorm error) of the cell-wise primal u against the exact solution."""
    nq = p + 3 if nq is None else nq
    out = np.zeros(2)
    lib().orc_error_norms(mesh.nx, mesh.ny, mesh.nz, _dp(mesh.verts), p, which, nq, _dp(_f64(u_cell)),
                          _dp(out))
    return float(out[0]), float(out[1])


def node_coords(mesh, p):
    xyz = np.zeros((mesh.ncells * (p + 1) ** 3, 3))
    lib().orc_node_coords(mesh.nx, mesh.ny, mesh.nz, _dp(mesh.verts), p, _dp(xyz))
    return xyz


def boundary_mask_global(mesh, p):
    """1 on interior global DoFs, 0 on DoFs of the boundary of the unit cube (homogeneous Dirichlet)."""
    gx, gy, gz = mesh.nx * p + 1, mesh.ny * p + 1, mesh.nz * p + 1
    k, j, i = np.meshgrid(np.arange(gz), np.arange(gy), np.arange(gx), indexing="ij")
    inner = (i > 0) & (i < gx - 1) & (j > 0) & (j < gy - 1) & (k > 0) & (k < gz - 1)
    return inner.astype(np.float64).ravel()


# ------------------------------------------------------ assembled problem
def assemble_global(mesh, p, kind):
    """A_CG = sum_K P_K^T A_K P_K as a scipy CSR matrix (brute force; tiny meshes only)."""
    import scipy.sparse as sp
    n3 = (p + 1) ** 3
    A = all_element_matrices(mesh, p, kind)
    gmap = global_index(mesh, p).reshape(mesh.ncells, n3)
    rows = np.repeat(gmap, n3, axis=1).ravel()
    cols = np.tile(gmap, (1, n3)).ravel()
    N = global_len(mesh, p)
    return sp.coo_matrix((A.ravel(), (rows, cols)), shape=(N, N)).tocsr()


def pcg_assembled(A, b, mask, tol=1e-10, maxit=10000, record=False):
    """Jacobi-preconditioned CG on the interior DoFs of the assembled system A u = b, u = 0 on the
    boundary. Stops when ||mask*(b - A u)|| <= tol * ||mask*b||. Returns (u, iterations, relres,
    iterates) where iterates[k] is u after k iterations when ``record``."""
    d = A.diagonal()
    dinv = np.where(mask > 0, 1.0 / d, 0.0)
    u = np.zeros_like(b)
    r = mask * b
    z = dinv * r
    p_ = z.copy()
    rho = r @ z
    nb = np.linalg.norm(mask * b)
    its = [u.copy()] if record else None
    k = 0
    relres = np.linalg.norm(r) / nb
    while k < maxit and relres > tol:
        q = mask * (A @ p_)
        alpha = rho / (p_ @ q)
        u = u + alpha * p_
        r = r - alpha * q
        z = dinv * r
        rho_new = r @ z
        p_ = z + (rho_new / rho) * p_
        rho = rho_new
        k += 1
        relres = np.linalg.norm(r) / nb
        if record:
            its.append(u.copy())
    return u, k, relres, its


def direct_solve(A, b, mask):
    """Sparse direct solve on the interior DoFs; boundary entries 0."""
    import scipy.sparse.linalg as spla
    idx = np.nonzero(mask > 0)[0]
    Aii = A[idx][:, idx].tocsc()
    u = np.zeros_like(b)
    u[idx] = spla.spsolve(Aii, b[idx])
    return u
