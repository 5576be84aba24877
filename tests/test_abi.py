"""The C-ABI library loads and exports every symbol that include/cwfem.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cwfem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cw_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_03413_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def declared_constants():
    src = open(os.path.join(ROOT, "include", "cwfem.h")).read()
    consts = {m.group(1): int(m.group(2), 0)
              for m in re.finditer(r"^#define (CW_[A-Z0-9_]+) (0x[0-9a-fA-F]+|\d+)", src, re.M)}
    consts.update({m.group(1): int(m.group(2)) for m in re.finditer(r"^\s+(CW_[A-Z_]+) = (\d+)", src, re.M)})
    return consts


def test_binding_constants_match_the_header():
    import paper_2607_03413_gb300 as pkg
    consts = declared_constants()
    assert len(consts) >= 30
    for name, value in consts.items():
        assert getattr(pkg, name) == value, name


def test_header_declares_the_binding_names():
    import paper_2607_03413_gb300 as pkg
    assert declared_functions() == sorted(pkg.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_and_argument_errors(lib):
    import paper_2607_03413_gb300 as pkg
    L = pkg.load()
    assert L.cw_status_string(0) == b"CW_OK"
    assert L.cw_status_string(7) == b"CW_ERR_UNSUPPORTED"
    # host-side argument checks run before any CUDA call
    assert L.cw_mesh_create(0, 1, 1, None, None) == pkg.CW_ERR_ARG
    h = ctypes.c_void_p()
    assert L.cw_mesh_create(2, 2, 2, None, ctypes.byref(h)) == pkg.CW_ERR_ARG
    assert L.cw_op_create(None, 2, 1, 1, 0, 0, ctypes.byref(h)) == pkg.CW_ERR_ARG
    assert L.cw_apply(None, None, None, 0, None) == pkg.CW_ERR_ARG
    assert L.cw_op_cellwise_len(None) == -1
    assert b"NULL" in L.cw_last_error()


def test_box_mesh_argument_errors(lib):
    import paper_2607_03413_gb300 as pkg
    L = pkg.load()
    h = ctypes.c_void_p()
    assert L.cw_mesh_create_box(0, 2, 2, 0.1, None, None, ctypes.byref(h)) == pkg.CW_ERR_ARG
    zero = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    assert L.cw_mesh_create_box(2, 2, 2, 0.1, None, ctypes.cast(zero, ctypes.c_void_p), ctypes.byref(h)) == pkg.CW_ERR_ARG
    assert L.cw_mesh_create_box(2, 2, 2, float("nan"), None, None, ctypes.byref(h)) == pkg.CW_ERR_ARG


def test_mesh_size_limits(lib):
    """At most 65535 cells per direction and 2^31 cells: rejected on the host before any device call."""
    import paper_2607_03413_gb300 as pkg
    L = pkg.load()
    h = ctypes.c_void_p()
    dummy = (ctypes.c_double * 3)()
    for dims in ((65536, 1, 1), (1, 65536, 1), (1, 1, 65536), (2 ** 31 - 1, 1, 1), (2048, 2048, 1024)):
        assert L.cw_mesh_create(*dims, ctypes.cast(dummy, ctypes.c_void_p), ctypes.byref(h)) == pkg.CW_ERR_ARG, dims
        assert L.cw_mesh_create_box(*dims, 0.0, None, None, ctypes.byref(h)) == pkg.CW_ERR_ARG, dims
        assert not h.value


def test_binding_checks_vector_lengths_and_dtypes():
    """The Python wrappers reject a vector of the wrong length or dtype before the C call, which
    could not tell (it takes bare pointers). Host-only: the checks run before any device work."""
    import torch
    import paper_2607_03413_gb300 as cw
    op = cw.Operator.__new__(cw.Operator)  # no library handle: the checks must fire first
    op.handle, op.L, op.NG, op.prec = None, 10, 27, cw.CW_PREC_F32
    good = torch.zeros(10, dtype=torch.float32)
    with pytest.raises(ValueError):
        op.apply(torch.zeros(9, dtype=torch.float32))
    with pytest.raises(TypeError):
        op.apply(torch.zeros(10, dtype=torch.float64))
    with pytest.raises(ValueError):
        op.apply(good, torch.zeros(11, dtype=torch.float32))
    with pytest.raises(ValueError):
        op.dss(torch.zeros(20, dtype=torch.float32))
    with pytest.raises(TypeError):  # the global input is FP64 whatever the storage precision
        op.gather(torch.zeros(27, dtype=torch.float32), good)
    with pytest.raises(ValueError):
        op.gather(torch.zeros(26, dtype=torch.float64), good)
    with pytest.raises(TypeError):  # solver vectors are FP64
        op.cg_solve(good)
    with pytest.raises(ValueError):
        op.cg_solve(torch.zeros(10, dtype=torch.float64), torch.zeros(5, dtype=torch.float64))
    with pytest.raises(ValueError):  # a batch's vectors hold nrhs cell-wise vectors
        cw.Batch([op], [2], [good], [good])
    with pytest.raises(ValueError):
        cw.Batch([op], [1, 1], [good], [good])
    with pytest.raises(TypeError):
        cw.Batch([op], [1], [good], [torch.zeros(10, dtype=torch.bfloat16)])


@pytest.mark.parametrize("perturb", [0.0, 0.3])
def test_mesh_refine_vertices_host(lib, perturb):
    """cw_mesh_refine_vertices (host only) gives the input generator's refinement bit for bit: the
    old vertices kept, midpoints of neighbours inserted axis by axis (pinned by closed forms in the
    multigrid oracle tests)."""
    import numpy as np

    import paper_2607_03413_gb300 as pkg
    import synth
    m = synth.box_mesh(3, 2, 4, perturb=perturb)
    out = pkg.cw_mesh_refine_vertices(m.nx, m.ny, m.nz, m.verts)
    assert np.array_equal(out, synth.refine(m).verts)
    twice = pkg.cw_mesh_refine_vertices(6, 4, 8, out)
    assert np.array_equal(twice, synth.refine(synth.refine(m)).verts)
    L = pkg.load()
    dummy = (ctypes.c_double * 3)()
    p = ctypes.cast(dummy, ctypes.c_void_p)
    assert L.cw_mesh_refine_vertices(40000, 1, 1, p, p) == pkg.CW_ERR_ARG  # 80000 cells in x
    assert L.cw_mesh_refine_vertices(1, 1, 1, None, p) == pkg.CW_ERR_ARG


def test_tune_cache_round_trip_and_replay(tmp_path, monkeypatch):
    """The JSON tuning cache: atomic save, reload, foreign files ignored; a cache hit sets the stored
    variant without timing, a miss times once and stores the choice (tuner calls faked on the host)."""
    import json

    import torch

    import paper_2607_03413_gb300 as cw
    from paper_2607_03413_gb300 import tune_cache
    path = tmp_path / "tune.json"
    tc = tune_cache.TuneCache(str(path))
    assert tc.entries == {}
    tc.put(tc.key("op", "dev", 4, 3), {"cells_per_cta": 0, "stage": 2, "ms": 1.5})
    assert json.loads(path.read_text())["entries"] and not list(tmp_path.glob("*.tmp*"))
    assert tune_cache.TuneCache(str(path)).get(tc.key("op", "dev", 4, 3))["stage"] == 2
    path.write_text("not json")
    assert tune_cache.TuneCache(str(path)).entries == {}

    calls = []
    monkeypatch.setattr(tune_cache, "device_name", lambda: "fake-gpu")
    monkeypatch.setattr(cw, "cw_op_autotune", lambda h, x, y, reps: calls.append("tune") or 0.25)
    monkeypatch.setattr(cw, "cw_op_get_variant", lambda h: (16, 2, (8, 16)))
    monkeypatch.setattr(cw, "cw_op_set_variant", lambda h, c, s: calls.append(("set", c, s)))
    op = cw.Operator.__new__(cw.Operator)
    op.handle, op.L, op.NG, op.prec = None, 10, 27, cw.CW_PREC_F64
    op.degree, op.kind, op.geom = 4, cw.CW_LAPLACE_MASS, cw.CW_GEOM_METRIC
    x = torch.zeros(10, dtype=torch.float64)
    y = torch.zeros(10, dtype=torch.float64)
    path2 = str(tmp_path / "ops.json")
    assert op.autotune(x, y, cache=path2) == 0.25 and calls == ["tune"]
    assert op.autotune(x, y, cache=path2) == 0.25 and calls == ["tune", ("set", 16, 2)]
    op.L = 20  # another size is another entry
    with pytest.raises(ValueError):
        op.autotune(x, y, cache=path2)  # (vectors of the old length are rejected first)
    x2, y2 = torch.zeros(20, dtype=torch.float64), torch.zeros(20, dtype=torch.float64)
    op.autotune(x2, y2, cache=path2)
    assert calls[-1] == "tune" and len(tune_cache.TuneCache(path2).entries) == 2


def test_batch_tune_cache_replay(tmp_path, monkeypatch):
    """Batch.autotune with a cache: the per-degree variants of a batch composition are stored after
    one timing run and set again without timing (tuner calls faked on the host)."""
    import types

    import paper_2607_03413_gb300 as cw
    from paper_2607_03413_gb300 import tune_cache
    calls = []
    monkeypatch.setattr(tune_cache, "device_name", lambda: "fake-gpu")
    monkeypatch.setattr(cw, "cw_batch_autotune", lambda h, reps: calls.append("tune") or 3.0)
    monkeypatch.setattr(cw, "cw_batch_get_variant", lambda h, d: ({2: 4, 5: 1}[d], 8))
    monkeypatch.setattr(cw, "cw_batch_set_variant", lambda h, d, v: calls.append(("set", d, v)))
    B = cw.Batch.__new__(cw.Batch)
    B.handle, B.mode, B.nrhs = None, cw.CW_BATCH_GROUPED, [2, 1, 1]
    B.ops = [types.SimpleNamespace(degree=d, kind=1, prec=0, L=L) for d, L in ((5, 100), (2, 27), (2, 54))]
    path = str(tmp_path / "batch.json")
    assert B.autotune(cache=path) == 3.0 and calls == ["tune"]
    calls.clear()
    assert B.autotune(cache=path) == 3.0
    assert sorted(calls) == [("set", 2, 4), ("set", 5, 1)]
    B.handle = None  # nothing to destroy


@pytest.mark.parametrize("p", range(1, 8))
def test_library_rules_match_the_oracle(lib, orc, p):
    """The library's own 1D rules (long-double Newton, host only) against the oracle's pinned rules:
    the Gauss-Lobatto nodes of the layout and the Gauss rule of the operators."""
    import numpy as np

    import paper_2607_03413_gb300 as pkg
    gll, xq, wq = pkg.cw_rules_1d(p)
    x_ref, w_ref = orc.gauss(p + 1)
    assert np.abs(gll - orc.gll(p)).max() < 1e-15
    assert np.abs(xq - x_ref).max() < 1e-15 and np.abs(wq - w_ref).max() < 1e-15


def test_library_rules_argument_errors(lib):
    import paper_2607_03413_gb300 as pkg
    assert pkg.load().cw_rules_1d(0, None, None, None) == pkg.CW_ERR_ARG
    assert pkg.load().cw_rules_1d(8, None, None, None) == pkg.CW_ERR_ARG


@pytest.mark.parametrize("p", range(1, 8))
def test_library_basis_matrices_match_the_oracle(lib, orc, p):
    """The library's 1D matrices against the same quantities formed from the oracle's pinned
    primitives (Lagrange basis by the product formula, Gauss rule): basis and derivative at the Gauss
    points, the collocation derivative on the Gauss points, the 1D mass and stiffness matrices."""
    import numpy as np

    import paper_2607_03413_gb300 as pkg
    B, Bd, D, M1, K1 = pkg.cw_basis_1d(p)
    xi = orc.gll(p)
    xq, wq = orc.gauss(p + 1)
    LB = np.array([orc.lagrange(xi, x)[0] for x in xq])
    LBd = np.array([orc.lagrange(xi, x)[1] for x in xq])
    LD = np.array([orc.lagrange(xq, x)[1] for x in xq])
    assert np.abs(B - LB).max() < 1e-13 and np.abs(Bd - LBd).max() < 1e-12
    assert np.abs(D - LD).max() < 1e-11
    assert np.abs(M1 - LB.T @ np.diag(wq) @ LB).max() < 1e-14
    assert np.abs(K1 - LBd.T @ np.diag(wq) @ LBd).max() < 1e-12 * max(1.0, np.abs(K1).max())


def test_entry_points_open_balanced_nvtx_ranges(lib, tmp_path):
    """Tracing: every entry point pushes an NVTX range "cwfem:<name>" and pops it on every return
    path (here the argument-error returns, which need no GPU). A small NVTX injection library
    (tests/nvtx_record.c, loaded by NVTX through NVTX_INJECTION64_PATH) records the ranges."""
    import shutil
    import subprocess
    import sys
    from paper_2607_03413_gb300 import build
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(build._nvcc())), "include")
    gcc = shutil.which("gcc") or pytest.skip("no gcc")
    rec = str(tmp_path / "libnvtx_record.so")
    subprocess.run([gcc, "-shared", "-fPIC", "-O1", "-I", cuda_inc, os.path.join(ROOT, "tests", "nvtx_record.c"),
                    "-o", rec], check=True)
    log = tmp_path / "ranges.txt"
    script = (
        "import paper_2607_03413_gb300 as pkg\n"
        "L = pkg.load()\n"
        "E = pkg.CW_ERR_ARG\n"
        "assert L.cw_apply(None, None, None, 0, None) == E\n"
        "assert L.cw_cg_solve(None, None, None, 1e-8, 10, 0, None, None) == E\n"
        "assert L.cw_mg_vcycle(None, None, None, 0, None) == E\n"
        "assert L.cw_mblock_apply(None, None, None, 0, None) == E\n"
    )
    env = dict(os.environ, NVTX_INJECTION64_PATH=rec, NVTX_RECORD_FILE=str(log), PYTHONPATH=ROOT)
    subprocess.run([sys.executable, "-c", script], check=True, env=env, cwd=ROOT, timeout=120)
    lines = log.read_text().split("\n")[:-1]
    assert lines == ["push cwfem:cw_apply", "pop", "push cwfem:cw_cg_solve", "pop",
                     "push cwfem:cw_mg_vcycle", "pop", "push cwfem:cw_mblock_apply", "pop"]
