"""Python binding of libcwfem.so, the sm_103a library for matrix-free high-order FEM operators on
cell-wise storage (apply, direct stiffness summation, Jacobi-PCG / mixed-precision refined CG).

This module only marshals arguments: every step of the computation runs in the library's CUDA
kernels. PyTorch tensors serve as device memory (``tensor.data_ptr()``) and streams
(``torch.cuda.current_stream().cuda_stream``). There is no CPU fallback: if the compiled library
is missing, loading fails with an error.

The functions ``cw_*`` have the names and argument order of ``include/cwfem.h``; ``Mesh`` and
``Operator`` hold handles and take tensors.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcwfem.so")

# constants mirrored from include/cwfem.h
CW_OK, CW_ERR_ARG, CW_ERR_OOM, CW_ERR_CUDA = 0, 1, 2, 3
CW_ERR_NOT_CONVERGED, CW_ERR_BREAKDOWN, CW_ERR_TIMEOUT, CW_ERR_UNSUPPORTED = 4, 5, 6, 7
CW_LAPLACE, CW_MASS, CW_LAPLACE_MASS = 1, 2, 3
CW_GEOM_AFFINE, CW_GEOM_METRIC, CW_GEOM_RECOMPUTE = 0, 1, 2
CW_PREC_F64, CW_PREC_F64_NATIVE, CW_PREC_F32, CW_PREC_F32_BF16G, CW_PREC_BF16 = 0, 1, 2, 3, 4
CW_BC_NONE, CW_BC_DIRICHLET0 = 0, 1
CW_APPLY_LOCAL, CW_APPLY_ASSEMBLE = 0, 1
CW_DSS_SUM, CW_DSS_AVERAGE = 0, 1
CW_CG_F64, CW_CG_IR_F32, CW_CG_IR_BF16, CW_CG_F64_NATIVE = 0, 1, 2, 3
CW_CG_WARM_START = 0x100
CW_BATCH_GROUPED, CW_BATCH_SINGLE = 0, 1

# exported symbols declared in include/cwfem.h (checked by the CPU test suite)
EXPORTED = [
    "cw_status_string", "cw_last_error", "cw_mesh_create", "cw_mesh_create_box", "cw_mesh_destroy", "cw_op_create",
    "cw_op_destroy", "cw_op_cellwise_len", "cw_op_global_len", "cw_op_device_bytes", "cw_gather",
    "cw_apply", "cw_dss", "cw_diagonal", "cw_load_vector", "cw_cg_solve", "cw_op_set_variant",
    "cw_op_get_variant", "cw_op_autotune", "cw_cg_solve_noalloc", "cw_batch_create", "cw_batch_destroy",
    "cw_batch_values", "cw_batch_launch", "cw_batch_graph_launch", "cw_batch_set_variant",
    "cw_batch_get_variant", "cw_batch_autotune", "cw_batch_set_mode", "cw_apply_batched", "cw_apply_host",
    "cw_mesh_refine_vertices", "cw_rules_1d", "cw_basis_1d", "cw_cg_residual", "cw_mg_create", "cw_mg_destroy",
    "cw_mg_device_bytes", "cw_mg_vcycle", "cw_mg_prolong", "cw_mg_restrict", "cw_mg_smooth", "cw_mg_coarse_solve",
    "cw_mg_pcg_solve", "cw_op_check", "cw_op_inject_stall", "cw_mblock_create", "cw_mblock_destroy",
    "cw_mblock_cellwise_len", "cw_mblock_global_len", "cw_mblock_shared_dofs", "cw_mblock_global_index",
    "cw_mblock_dss", "cw_mblock_apply", "cw_mblock_diagonal", "cw_mblock_cg_solve",
]


class CwError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.cw_last_error().decode() if _lib is not None else ""
        super().__init__(f"{where}: {_lib.cw_status_string(status).decode()} {msg}")


class cw_cg_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer_iterations", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("energy", ctypes.c_double),
                ("seconds", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libcwfem.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libcwfem.so not found at {path}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "cw_status_string": ([i32], ctypes.c_char_p),
        "cw_last_error": ([], ctypes.c_char_p),
        "cw_mesh_create": ([i32, i32, i32, vp, ctypes.POINTER(vp)], i32),
        "cw_mesh_create_box": ([i32, i32, i32, ctypes.c_double, vp, vp, ctypes.POINTER(vp)], i32),
        "cw_mesh_destroy": ([vp], i32),
        "cw_op_create": ([vp, i32, i32, i32, i32, i32, ctypes.POINTER(vp)], i32),
        "cw_op_destroy": ([vp], i32),
        "cw_op_cellwise_len": ([vp], i64),
        "cw_op_global_len": ([vp], i64),
        "cw_op_device_bytes": ([vp], i64),
        "cw_gather": ([vp, vp, vp, vp], i32),
        "cw_apply": ([vp, vp, vp, i32, vp], i32),
        "cw_dss": ([vp, vp, i32, vp], i32),
        "cw_diagonal": ([vp, vp, vp], i32),
        "cw_load_vector": ([vp, i32, vp, vp], i32),
        "cw_cg_solve": ([vp, vp, vp, dbl, i32, i32, ctypes.POINTER(cw_cg_stats), vp], i32),
        "cw_op_set_variant": ([vp, i32, i32], i32),
        "cw_op_get_variant": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)], i32),
        "cw_op_autotune": ([vp, vp, vp, i32, vp, ctypes.POINTER(ctypes.c_float)], i32),
        "cw_cg_solve_noalloc": ([vp, vp, vp, dbl, i32, i32, ctypes.POINTER(cw_cg_stats), vp], i32),
        "cw_batch_create": ([ctypes.POINTER(vp), ctypes.POINTER(i32), ctypes.POINTER(vp), ctypes.POINTER(vp), i32,
                             ctypes.POINTER(vp)], i32),
        "cw_batch_destroy": ([vp], i32),
        "cw_batch_values": ([vp], i64),
        "cw_batch_launch": ([vp, vp], i32),
        "cw_batch_graph_launch": ([vp, vp], i32),
        "cw_batch_set_variant": ([vp, i32, i32], i32),
        "cw_batch_get_variant": ([vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)], i32),
        "cw_batch_autotune": ([vp, i32, vp, ctypes.POINTER(ctypes.c_float)], i32),
        "cw_batch_set_mode": ([vp, i32], i32),
        "cw_apply_batched": ([ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i32), i32,
                              i32, vp], i32),
        "cw_apply_host": ([vp, vp, vp, i32, vp], i32),
        "cw_mesh_refine_vertices": ([i32, i32, i32, vp, vp], i32),
        "cw_rules_1d": ([i32, vp, vp, vp], i32),
        "cw_basis_1d": ([i32, vp, vp, vp, vp, vp], i32),
        "cw_cg_residual": ([vp, vp, vp, i32, ctypes.POINTER(dbl), vp], i32),
        "cw_op_check": ([vp, vp], i32),
        "cw_mblock_create": ([ctypes.POINTER(vp), i32, ctypes.POINTER(vp)], i32),
        "cw_mblock_destroy": ([vp], i32),
        "cw_mblock_cellwise_len": ([vp], i64),
        "cw_mblock_global_len": ([vp], i64),
        "cw_mblock_shared_dofs": ([vp, i32], i64),
        "cw_mblock_global_index": ([vp, vp], i32),
        "cw_mblock_dss": ([vp, vp, i32, vp], i32),
        "cw_mblock_apply": ([vp, vp, vp, i32, vp], i32),
        "cw_mblock_diagonal": ([vp, vp, vp], i32),
        "cw_mblock_cg_solve": ([vp, vp, vp, dbl, i32, ctypes.POINTER(cw_cg_stats), vp], i32),
        "cw_op_inject_stall": ([vp, i32], i32),
        "cw_mg_create": ([ctypes.POINTER(vp), i32, i32, i32, dbl, ctypes.POINTER(vp)], i32),
        "cw_mg_destroy": ([vp], i32),
        "cw_mg_device_bytes": ([vp], i64),
        "cw_mg_vcycle": ([vp, vp, vp, i32, vp], i32),
        "cw_mg_prolong": ([vp, i32, vp, vp, vp], i32),
        "cw_mg_restrict": ([vp, i32, vp, vp, vp], i32),
        "cw_mg_smooth": ([vp, i32, vp, vp, i32, vp], i32),
        "cw_mg_coarse_solve": ([vp, vp, vp, vp], i32),
        "cw_mg_pcg_solve": ([vp, vp, vp, vp, dbl, i32, ctypes.POINTER(cw_cg_stats), vp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(st, where):
    if st != CW_OK:
        raise CwError(st, where)


def _stream(stream=None):
    if stream is not None:
        return ctypes.c_void_p(stream)
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if hasattr(t, "is_cuda") and not t.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(int(t))


# ------------------------------------------------------------------ C-ABI mirrors ----
def cw_mesh_create(nx, ny, nz, verts_host):
    import numpy as np
    L = load()
    v = np.ascontiguousarray(verts_host, dtype=np.float64)
    assert v.size == (nx + 1) * (ny + 1) * (nz + 1) * 3
    h = ctypes.c_void_p()
    _check(L.cw_mesh_create(nx, ny, nz, v.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)), "cw_mesh_create")
    return h


def cw_mesh_create_box(nx, ny, nz, perturb=0.0, freq=None, direction=None):
    L = load()
    f = (ctypes.c_int * 3)(*freq) if freq is not None else None
    d = (ctypes.c_double * 3)(*direction) if direction is not None else None
    h = ctypes.c_void_p()
    _check(L.cw_mesh_create_box(nx, ny, nz, float(perturb), ctypes.cast(f, ctypes.c_void_p) if f else None,
                                ctypes.cast(d, ctypes.c_void_p) if d else None, ctypes.byref(h)),
           "cw_mesh_create_box")
    return h


def cw_mesh_refine_vertices(nx, ny, nz, verts):
    """Vertex array [(2nz+1),(2ny+1),(2nx+1),3] of the uniform refinement (host only)."""
    import numpy as np
    v = np.ascontiguousarray(verts, dtype=np.float64)
    assert v.size == (nx + 1) * (ny + 1) * (nz + 1) * 3
    out = np.empty((2 * nz + 1, 2 * ny + 1, 2 * nx + 1, 3))
    _check(load().cw_mesh_refine_vertices(nx, ny, nz, v.ctypes.data_as(ctypes.c_void_p),
                                          out.ctypes.data_as(ctypes.c_void_p)), "cw_mesh_refine_vertices")
    return out


def cw_rules_1d(degree):
    """(Gauss-Lobatto nodes, Gauss points, Gauss weights) on [0, 1], p+1 each (host only)."""
    import numpy as np
    out = [np.empty(degree + 1) for _ in range(3)]
    _check(load().cw_rules_1d(degree, *[a.ctypes.data_as(ctypes.c_void_p) for a in out]), "cw_rules_1d")
    return tuple(out)


def cw_basis_1d(degree):
    """(B, Bd, D, M1, K1), each (p+1) x (p+1): basis and derivative at the Gauss points, collocation
    derivative on the Gauss points, 1D mass and stiffness matrices (host only)."""
    import numpy as np
    n = degree + 1
    out = [np.empty((n, n)) for _ in range(5)]
    _check(load().cw_basis_1d(degree, *[a.ctypes.data_as(ctypes.c_void_p) for a in out]), "cw_basis_1d")
    return tuple(out)


def cw_mesh_destroy(h):
    _check(load().cw_mesh_destroy(h), "cw_mesh_destroy")


def cw_op_create(mesh, degree, kind, geom, prec, bc=CW_BC_NONE):
    h = ctypes.c_void_p()
    _check(load().cw_op_create(mesh, degree, kind, geom, prec, bc, ctypes.byref(h)), "cw_op_create")
    return h


def cw_op_destroy(h):
    _check(load().cw_op_destroy(h), "cw_op_destroy")


def cw_op_cellwise_len(h):
    return load().cw_op_cellwise_len(h)


def cw_op_global_len(h):
    return load().cw_op_global_len(h)


def cw_op_device_bytes(h):
    return load().cw_op_device_bytes(h)


def cw_gather(op, u_global, x, stream=None):
    _check(load().cw_gather(op, _ptr(u_global), _ptr(x), _stream(stream)), "cw_gather")


def cw_apply(op, x, y, flags=CW_APPLY_LOCAL, stream=None):
    _check(load().cw_apply(op, _ptr(x), _ptr(y), flags, _stream(stream)), "cw_apply")


def _host_ptr(t):
    if hasattr(t, "data_ptr"):
        if getattr(t, "is_cuda", False):
            raise ValueError("expected a host (CPU) tensor")
        if not t.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)


def cw_apply_host(op, x_host, y_host, flags=CW_APPLY_LOCAL, stream=None):
    _check(load().cw_apply_host(op, _host_ptr(x_host), _host_ptr(y_host), flags, _stream(stream)), "cw_apply_host")


def cw_dss(op, v, flags=CW_DSS_SUM, stream=None):
    _check(load().cw_dss(op, _ptr(v), flags, _stream(stream)), "cw_dss")


def cw_diagonal(op, d, stream=None):
    _check(load().cw_diagonal(op, _ptr(d), _stream(stream)), "cw_diagonal")


def cw_load_vector(op, which, b, stream=None):
    _check(load().cw_load_vector(op, which, _ptr(b), _stream(stream)), "cw_load_vector")


def cw_cg_solve(op, b, u, rtol=1e-10, maxit=10000, mode=CW_CG_F64, stream=None, check=True):
    st = cw_cg_stats()
    rc = load().cw_cg_solve(op, _ptr(b), _ptr(u), rtol, maxit, mode, ctypes.byref(st), _stream(stream))
    if check and rc not in (CW_OK,):
        raise CwError(rc, "cw_cg_solve")
    return rc, st


def cw_cg_residual(op, b, u, prec=CW_PREC_F64_NATIVE, stream=None):
    """Relative residual ||m G^T(b - A u)|| / ||m G^T b|| with A in precision ``prec``
    (CW_PREC_F64_NATIVE: the IEEE FP64 operator; CW_PREC_F64: double-float on the float-pair metric)."""
    r = ctypes.c_double()
    _check(load().cw_cg_residual(op, _ptr(b), _ptr(u), prec, ctypes.byref(r), _stream(stream)), "cw_cg_residual")
    return r.value


def cw_cg_solve_noalloc(op, b, u, rtol=1e-10, maxit=10000, mode=CW_CG_F64, stream=None):
    """Allocation-free FP64 solve (fixed library-owned scratch, cell-wise length <= 2^18)."""
    st = cw_cg_stats()
    rc = load().cw_cg_solve_noalloc(op, _ptr(b), _ptr(u), rtol, maxit, mode, ctypes.byref(st), _stream(stream))
    return rc, st


def cw_op_check(op, stream=None):
    """CW_OK, or CW_ERR_TIMEOUT if a bounded wait of the operator's kernels expired since the last check."""
    return load().cw_op_check(op, _stream(stream))


def cw_op_inject_stall(op, on=True):
    _check(load().cw_op_inject_stall(op, int(bool(on))), "cw_op_inject_stall")


def cw_op_set_variant(op, cells_per_cta, stage):
    _check(load().cw_op_set_variant(op, cells_per_cta, stage), "cw_op_set_variant")


def cw_op_get_variant(op):
    c, s, ch = ctypes.c_int(), ctypes.c_int(), (ctypes.c_int * 2)()
    _check(load().cw_op_get_variant(op, ctypes.byref(c), ctypes.byref(s), ch), "cw_op_get_variant")
    return c.value, s.value, (ch[0], ch[1])


def cw_op_autotune(op, x, y, reps=5, stream=None):
    ms = ctypes.c_float()
    _check(load().cw_op_autotune(op, _ptr(x), _ptr(y), reps, _stream(stream), ctypes.byref(ms)), "cw_op_autotune")
    return ms.value


def cw_batch_create(ops, nrhs, xs, ys):
    n = len(ops)
    VP = ctypes.c_void_p * n
    h = ctypes.c_void_p()
    _check(load().cw_batch_create(VP(*[o.value if isinstance(o, ctypes.c_void_p) else o for o in ops]),
                                  (ctypes.c_int * n)(*nrhs), VP(*[_ptr(x).value for x in xs]),
                                  VP(*[_ptr(y).value for y in ys]), n, ctypes.byref(h)), "cw_batch_create")
    return h


def cw_batch_destroy(b):
    _check(load().cw_batch_destroy(b), "cw_batch_destroy")


def cw_batch_values(b):
    return load().cw_batch_values(b)


def cw_batch_launch(b, stream=None):
    _check(load().cw_batch_launch(b, _stream(stream)), "cw_batch_launch")


def cw_batch_graph_launch(b, stream=None):
    _check(load().cw_batch_graph_launch(b, _stream(stream)), "cw_batch_graph_launch")


def cw_batch_set_mode(b, mode):
    _check(load().cw_batch_set_mode(b, mode), "cw_batch_set_mode")


def cw_batch_set_variant(b, degree, variant):
    _check(load().cw_batch_set_variant(b, degree, variant), "cw_batch_set_variant")


def cw_batch_get_variant(b, degree):
    h, c = ctypes.c_int(), ctypes.c_int()
    _check(load().cw_batch_get_variant(b, degree, ctypes.byref(h), ctypes.byref(c)), "cw_batch_get_variant")
    return h.value, c.value


def cw_batch_autotune(b, reps=3, stream=None):
    ms = ctypes.c_float()
    _check(load().cw_batch_autotune(b, reps, _stream(stream), ctypes.byref(ms)), "cw_batch_autotune")
    return ms.value


def cw_apply_batched(ops, xs, ys, nrhs, flags=CW_APPLY_LOCAL, stream=None):
    n = len(ops)
    VP = ctypes.c_void_p * n
    _check(load().cw_apply_batched(VP(*[o.value if isinstance(o, ctypes.c_void_p) else o for o in ops]),
                                   VP(*[_ptr(x).value for x in xs]), VP(*[_ptr(y).value for y in ys]),
                                   (ctypes.c_int * n)(*nrhs), n, flags, _stream(stream)), "cw_apply_batched")


def cw_mg_create(ops, nu1=2, nu2=2, omega=0.7):
    n = len(ops)
    h = ctypes.c_void_p()
    _check(load().cw_mg_create((ctypes.c_void_p * n)(*[o.value if isinstance(o, ctypes.c_void_p) else o for o in ops]),
                               n, nu1, nu2, float(omega), ctypes.byref(h)), "cw_mg_create")
    return h


def cw_mg_destroy(mg):
    _check(load().cw_mg_destroy(mg), "cw_mg_destroy")


def cw_mg_device_bytes(mg):
    return load().cw_mg_device_bytes(mg)


def cw_mg_vcycle(mg, b, u, zero_guess=True, stream=None):
    _check(load().cw_mg_vcycle(mg, _ptr(b), _ptr(u), int(bool(zero_guess)), _stream(stream)), "cw_mg_vcycle")


def cw_mg_prolong(mg, level, uc, uf, stream=None):
    _check(load().cw_mg_prolong(mg, level, _ptr(uc), _ptr(uf), _stream(stream)), "cw_mg_prolong")


def cw_mg_restrict(mg, level, rf, rc, stream=None):
    _check(load().cw_mg_restrict(mg, level, _ptr(rf), _ptr(rc), _stream(stream)), "cw_mg_restrict")


def cw_mg_smooth(mg, level, b, u, sweeps=1, stream=None):
    _check(load().cw_mg_smooth(mg, level, _ptr(b), _ptr(u), sweeps, _stream(stream)), "cw_mg_smooth")


def cw_mg_coarse_solve(mg, b, u, stream=None):
    _check(load().cw_mg_coarse_solve(mg, _ptr(b), _ptr(u), _stream(stream)), "cw_mg_coarse_solve")


def cw_mg_pcg_solve(mg, op, b, u, rtol=1e-10, maxit=1000, stream=None, check=True):
    st = cw_cg_stats()
    rc = load().cw_mg_pcg_solve(mg, op, _ptr(b), _ptr(u), rtol, maxit, ctypes.byref(st), _stream(stream))
    if check and rc != CW_OK:
        raise CwError(rc, "cw_mg_pcg_solve")
    return rc, st


# ------------------------------------------------------------------ convenience ----
_VEC_DTYPE = {CW_PREC_F64: "float64", CW_PREC_F64_NATIVE: "float64", CW_PREC_F32: "float32",
              CW_PREC_F32_BF16G: "float32", CW_PREC_BF16: "bfloat16"}


def _vec(t, n, dtype, what):
    """Checks a vector argument against the length and dtype the C call assumes for it (the C ABI
    takes bare pointers and cannot see either)."""
    if t.dtype != dtype:
        raise TypeError(f"{what}: expected dtype {dtype}, got {t.dtype}")
    if t.numel() != n:
        raise ValueError(f"{what}: expected {n} values, got {t.numel()}")
    return t


class Mesh:
    """Owns a cw_mesh handle built from a vertex array [(nz+1),(ny+1),(nx+1),3]."""

    def __init__(self, nx, ny, nz, verts):
        import numpy as np
        self.nx, self.ny, self.nz = nx, ny, nz
        self.verts = np.ascontiguousarray(verts, dtype=np.float64)  # kept for refine()
        self.handle = cw_mesh_create(nx, ny, nz, self.verts)

    @classmethod
    def from_synth(cls, m):
        return cls(m.nx, m.ny, m.nz, m.verts)

    @classmethod
    def box(cls, nx, ny=None, nz=None, perturb=0.0, freq=None, direction=None):
        """The unit-cube box mesh generated by the library (cw_mesh_create_box)."""
        ny = nx if ny is None else ny
        nz = nx if nz is None else nz
        self = cls.__new__(cls)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.verts = None  # generated in the library
        self.handle = cw_mesh_create_box(nx, ny, nz, perturb, freq, direction)
        return self

    def refine(self):
        """The next level of a uniform hierarchy (every cell split into 2 x 2 x 2 by its trilinear map)."""
        if self.verts is None:
            raise ValueError("refine() needs a mesh built from a vertex array (Mesh(...) or from_synth)")
        return Mesh(2 * self.nx, 2 * self.ny, 2 * self.nz,
                    cw_mesh_refine_vertices(self.nx, self.ny, self.nz, self.verts))

    def close(self):
        if self.handle:
            cw_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Operator:
    """Owns a cw_op handle; methods take torch tensors on the current CUDA device."""

    def __init__(self, mesh: Mesh, degree, kind=CW_LAPLACE, geom=CW_GEOM_METRIC, prec=CW_PREC_F64,
                 bc=CW_BC_NONE):
        self.mesh = mesh
        self.degree, self.kind, self.geom, self.prec, self.bc = degree, kind, geom, prec, bc
        self.handle = cw_op_create(mesh.handle, degree, kind, geom, prec, bc)
        self.L = cw_op_cellwise_len(self.handle)
        self.NG = cw_op_global_len(self.handle)

    @property
    def vec_dtype(self):
        import torch
        return getattr(torch, _VEC_DTYPE[self.prec])

    def empty(self):
        import torch
        return torch.empty(self.L, dtype=self.vec_dtype, device="cuda")

    def _cw(self, t, what):  # a cell-wise vector in the operator's storage type
        return _vec(t, self.L, self.vec_dtype, what)

    def _f64(self, t, what):  # a cell-wise FP64 vector (diagonal, load vector, solver vectors)
        import torch
        return _vec(t, self.L, torch.float64, what)

    def gather(self, u_global, x=None):
        import torch
        _vec(u_global, self.NG, torch.float64, "gather: u_global")
        x = self.empty() if x is None else self._cw(x, "gather: x")
        cw_gather(self.handle, u_global, x)
        return x

    def apply(self, x, y=None, assemble=False):
        self._cw(x, "apply: x")
        y = self.empty() if y is None else self._cw(y, "apply: y")
        cw_apply(self.handle, x, y, CW_APPLY_ASSEMBLE if assemble else CW_APPLY_LOCAL)
        return y

    def set_variant(self, cells_per_cta=0, stage=1):
        cw_op_set_variant(self.handle, cells_per_cta, stage)

    def variant(self):
        return cw_op_get_variant(self.handle)

    def autotune(self, x, y, reps=5, cache=None):
        """Time every kernel variant and keep the fastest; returns its time per apply in ms. With a
        ``TuneCache`` (or a path to one) an earlier choice for the same device, operator and size is
        set without timing (the returned time is then the cached one)."""
        self._cw(x, "autotune: x")
        self._cw(y, "autotune: y")
        if cache is None:
            return cw_op_autotune(self.handle, x, y, reps)
        from .tune_cache import TuneCache, device_name
        tc = cache if isinstance(cache, TuneCache) else TuneCache(cache)
        key = tc.key("op", device_name(), self.degree, self.kind, self.geom, self.prec, self.L)
        hit = tc.get(key)
        if hit is not None:
            self.set_variant(hit["cells_per_cta"], hit["stage"])
            return hit["ms"]
        ms = cw_op_autotune(self.handle, x, y, reps)
        cpb, stage, choices = self.variant()
        # 0 = the degree's default tile (the only value some operators accept back)
        tc.put(key, {"cells_per_cta": 0 if cpb == choices[0] else cpb, "stage": stage, "ms": ms})
        return ms

    def dss(self, v, average=False):
        cw_dss(self.handle, self._cw(v, "dss: v"), CW_DSS_AVERAGE if average else CW_DSS_SUM)
        return v

    def diagonal(self):
        import torch
        d = torch.empty(self.L, dtype=torch.float64, device="cuda")
        cw_diagonal(self.handle, d)
        return d

    def load_vector(self, which=0):
        import torch
        b = torch.empty(self.L, dtype=torch.float64, device="cuda")
        cw_load_vector(self.handle, which, b)
        return b

    def cg_solve(self, b, u=None, rtol=1e-10, maxit=10000, mode=CW_CG_F64, check=True, warm_start=False):
        """Jacobi-PCG (cw_cg_solve); warm_start: start from the given u (resume an earlier solve)."""
        import torch
        self._f64(b, "cg_solve: b")
        if warm_start and u is None:
            raise ValueError("cg_solve: warm_start needs the initial iterate u")
        u = torch.empty(self.L, dtype=torch.float64, device="cuda") if u is None else self._f64(u, "cg_solve: u")
        rc, st = cw_cg_solve(self.handle, b, u, rtol, maxit, mode | (CW_CG_WARM_START if warm_start else 0),
                             check=check)
        return u, st, rc

    def residual(self, b, u, prec=CW_PREC_F64_NATIVE):
        """Relative residual of the solver's measure for iterate u (see cw_cg_residual)."""
        self._f64(b, "residual: b")
        self._f64(u, "residual: u")
        return cw_cg_residual(self.handle, b, u, prec)

    def close(self):
        if self.handle:
            cw_op_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owns a cw_batch handle; keeps references to its operators and vectors."""

    def __init__(self, ops, nrhs, xs, ys):
        self.ops, self.nrhs, self.xs, self.ys = list(ops), list(nrhs), list(xs), list(ys)
        if not (len(self.ops) == len(self.nrhs) == len(self.xs) == len(self.ys)):
            raise ValueError("Batch: ops, nrhs, xs and ys differ in length")
        for i, (o, r, x, y) in enumerate(zip(self.ops, self.nrhs, self.xs, self.ys)):
            _vec(x, r * o.L, o.vec_dtype, f"Batch: xs[{i}]")
            _vec(y, r * o.L, o.vec_dtype, f"Batch: ys[{i}]")
        self.handle = cw_batch_create([o.handle for o in self.ops], self.nrhs, self.xs, self.ys)
        self.values = cw_batch_values(self.handle)
        self.mode = CW_BATCH_GROUPED

    def launch(self, graph=False, stream=None):
        (cw_batch_graph_launch if graph else cw_batch_launch)(self.handle, stream)

    def autotune(self, reps=3, cache=None, mode=None):
        """Per-degree autotuning of the current mode (``mode`` sets it first); returns the batch time
        in ms. With a ``TuneCache`` (or a path) an earlier choice for the same device, mode and batch
        composition is set without timing."""
        if mode is not None:
            self.set_mode(mode)
        if cache is None:
            return cw_batch_autotune(self.handle, reps)
        from .tune_cache import TuneCache, device_name
        tc = cache if isinstance(cache, TuneCache) else TuneCache(cache)
        comp = sorted((o.degree, o.kind, o.prec, o.L, r) for o, r in zip(self.ops, self.nrhs))
        key = tc.key("batch", device_name(), self.mode, comp)
        hit = tc.get(key)
        if hit is not None:
            for degree, variant in hit["variants"].items():
                self.set_variant(int(degree), variant)
            return hit["ms"]
        ms = cw_batch_autotune(self.handle, reps)
        variants = {str(d): self.variant(d)[0] for d in sorted({o.degree for o in self.ops})}
        tc.put(key, {"variants": variants, "ms": ms})
        return ms

    def set_mode(self, mode):
        cw_batch_set_mode(self.handle, mode)
        self.mode = mode

    def set_variant(self, degree, variant):
        cw_batch_set_variant(self.handle, degree, variant)

    def variant(self, degree):
        return cw_batch_get_variant(self.handle, degree)

    def close(self):
        if self.handle:
            cw_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Multigrid:
    """Owns a cw_mg handle over a list of Operators (coarsest first); keeps references to them."""

    def __init__(self, ops, nu1=2, nu2=2, omega=0.7):
        self.ops = list(ops)
        self.nu1, self.nu2, self.omega = nu1, nu2, omega
        self.handle = cw_mg_create([o.handle for o in self.ops], nu1, nu2, omega)

    @property
    def top(self):
        return self.ops[-1]

    def vcycle(self, b, u=None, zero_guess=True):
        top = self.top
        top._cw(b, "vcycle: b")
        u = top.empty() if u is None else top._cw(u, "vcycle: u")
        cw_mg_vcycle(self.handle, b, u, zero_guess)
        return u

    def prolong(self, level, uc, uf=None):
        f, c = self.ops[level], self.ops[level - 1]
        c._cw(uc, "prolong: uc")
        uf = f.empty() if uf is None else f._cw(uf, "prolong: uf")
        cw_mg_prolong(self.handle, level, uc, uf)
        return uf

    def restrict(self, level, rf, rc=None):
        f, c = self.ops[level], self.ops[level - 1]
        f._cw(rf, "restrict: rf")
        rc = c.empty() if rc is None else c._cw(rc, "restrict: rc")
        cw_mg_restrict(self.handle, level, rf, rc)
        return rc

    def smooth(self, level, b, u, sweeps=1):
        o = self.ops[level]
        cw_mg_smooth(self.handle, level, o._cw(b, "smooth: b"), o._cw(u, "smooth: u"), sweeps)
        return u

    def coarse_solve(self, b, u=None):
        o = self.ops[0]
        o._cw(b, "coarse_solve: b")
        u = o.empty() if u is None else o._cw(u, "coarse_solve: u")
        cw_mg_coarse_solve(self.handle, b, u)
        return u

    def pcg_solve(self, op, b, u=None, rtol=1e-10, maxit=1000, check=True):
        """MG-preconditioned CG for the FP64 operator `op` on the finest level's mesh."""
        import torch
        op._f64(b, "pcg_solve: b")
        u = torch.empty(op.L, dtype=torch.float64, device="cuda") if u is None else op._f64(u, "pcg_solve: u")
        rc, st = cw_mg_pcg_solve(self.handle, op.handle, b, u, rtol, maxit, check=check)
        return u, st, rc

    def close(self):
        if self.handle:
            cw_mg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MultiBlock:
    """Owns a cw_mblock handle over per-block Operators (kept referenced); cell-wise vectors are the
    concatenation of the blocks' vectors."""

    def __init__(self, ops):
        self.ops = list(ops)
        n = len(self.ops)
        h = ctypes.c_void_p()
        _check(load().cw_mblock_create((ctypes.c_void_p * n)(*[o.handle.value for o in self.ops]), n, ctypes.byref(h)),
               "cw_mblock_create")
        self.handle = h
        self.L = load().cw_mblock_cellwise_len(h)
        self.NG = load().cw_mblock_global_len(h)
        self.vec_dtype = self.ops[0].vec_dtype

    def shared_dofs(self):
        return tuple(load().cw_mblock_shared_dofs(self.handle, s) for s in range(3))

    def global_index(self):
        import numpy as np
        out = np.empty(self.L, dtype=np.int64)
        _check(load().cw_mblock_global_index(self.handle, out.ctypes.data_as(ctypes.c_void_p)), "cw_mblock_global_index")
        return out

    def empty(self):
        import torch
        return torch.empty(self.L, dtype=self.vec_dtype, device="cuda")

    def dss(self, v, average=False):
        _vec(v, self.L, self.vec_dtype, "mblock dss: v")
        _check(load().cw_mblock_dss(self.handle, _ptr(v), CW_DSS_AVERAGE if average else CW_DSS_SUM, _stream(None)),
               "cw_mblock_dss")
        return v

    def apply(self, x, y=None, assemble=False):
        _vec(x, self.L, self.vec_dtype, "mblock apply: x")
        y = self.empty() if y is None else _vec(y, self.L, self.vec_dtype, "mblock apply: y")
        _check(load().cw_mblock_apply(self.handle, _ptr(x), _ptr(y), CW_APPLY_ASSEMBLE if assemble else CW_APPLY_LOCAL,
                                      _stream(None)), "cw_mblock_apply")
        return y

    def diagonal(self):
        import torch
        d = torch.empty(self.L, dtype=torch.float64, device="cuda")
        _check(load().cw_mblock_diagonal(self.handle, _ptr(d), _stream(None)), "cw_mblock_diagonal")
        return d

    def cg_solve(self, b, u=None, rtol=1e-10, maxit=10000, check=True):
        import torch
        _vec(b, self.L, torch.float64, "mblock cg_solve: b")
        u = torch.empty(self.L, dtype=torch.float64, device="cuda") if u is None else _vec(u, self.L, torch.float64, "u")
        st = cw_cg_stats()
        rc = load().cw_mblock_cg_solve(self.handle, _ptr(b), _ptr(u), rtol, maxit, ctypes.byref(st), _stream(None))
        if check and rc != CW_OK:
            raise CwError(rc, "cw_mblock_cg_solve")
        return u, st, rc

    def close(self):
        if self.handle:
            _check(load().cw_mblock_destroy(self.handle), "cw_mblock_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
