"""GPU parity of the sum-factorised apply, gather, DSS, diagonal and load vector against the FP64
oracle, through the C ABI. FP64 paths: ||y - y_ref||_inf / ||y_ref||_inf <= 1e-12."""
import numpy as np
import pytest

import synth
from gpu_util import rel_err, to_np

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


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


def mesh_for(p):
    # several tiles of every tile size plus a ragged last tile
    return synth.box_mesh(3, 4, 5, perturb=0.2) if p <= 5 else synth.box_mesh(3, 1, 3, perturb=0.2)


def run_apply(cw, mesh, p, kind, geom, prec, xin, assemble=False):
    import torch
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, p, kind, geom, prec)
    x = torch.from_numpy(xin).cuda().to(op.vec_dtype)
    y = op.apply(x, assemble=assemble)
    torch.cuda.synchronize()
    return to_np(y)


@pytest.mark.parametrize("prec", [0, 1], ids=["df64", "f64native"])
@pytest.mark.parametrize("kind", [1, 2, 3], ids=["K", "M", "KM"])
@pytest.mark.parametrize("p", range(1, 8))
def test_apply_metric_f64(cw, orc, p, kind, prec):
    mesh = mesh_for(p)
    x = orc.gather(mesh, p, synth.global_vector(mesh, p, seed=p))
    ref = orc.apply_local(mesh, p, kind, x)
    y = run_apply(cw, mesh, p, kind, cw.CW_GEOM_METRIC, prec, x)
    assert rel_err(y, ref) <= TOL64


@pytest.mark.parametrize("prec", [0, 1], ids=["df64", "f64native"])
@pytest.mark.parametrize("kind", [1, 2, 3], ids=["K", "M", "KM"])
@pytest.mark.parametrize("p", range(1, 8))
def test_apply_recompute_f64(cw, orc, p, kind, prec):
    """Metric recomputed at every quadrature point from the cell's trilinear coefficients: the same
    operator as the oracle's element matrices."""
    mesh = mesh_for(p)
    x = orc.gather(mesh, p, synth.global_vector(mesh, p, seed=50 + p))
    ref = orc.apply_local(mesh, p, kind, x)
    y = run_apply(cw, mesh, p, kind, cw.CW_GEOM_RECOMPUTE, prec, x)
    assert rel_err(y, ref) <= TOL64


@pytest.mark.parametrize("prec,tol", [(2, 2e-6), (3, 2e-6), (4, 3e-2)], ids=["f32", "f32_bf16g", "bf16"])
@pytest.mark.parametrize("p", [1, 3, 4, 7])
def test_apply_recompute_reduced_precision_error(cw, orc, p, prec, tol):
    """Recomputed geometry in FP32 arithmetic (coefficients stored as floats for every reduced
    precision): error against the FP64 oracle, bounded by the vector storage precision."""
    mesh = mesh_for(p)
    x = orc.gather(mesh, p, synth.global_vector(mesh, p, seed=p))
    ref = orc.apply_local(mesh, p, 3, x)
    y = run_apply(cw, mesh, p, 3, cw.CW_GEOM_RECOMPUTE, prec, x)
    err = rel_err(y, ref)
    print(f"p={p} prec={prec} rel err {err:.3e}")
    assert err <= tol


@pytest.mark.parametrize("kind", [1, 2, 3], ids=["K", "M", "KM"])
@pytest.mark.parametrize("p", range(1, 8))
def test_apply_affine_f64(cw, orc, p, kind):
    mesh = synth.box_mesh(5, 3, 4) if p <= 5 else synth.box_mesh(3, 2, 2)
    x = synth.cellwise_random(mesh, p, seed=10 + p)  # the apply is cell-local: any input works
    ref = orc.apply_local(mesh, p, kind, x)
    y = run_apply(cw, mesh, p, kind, cw.CW_GEOM_AFFINE, cw.CW_PREC_F64, x)
    assert rel_err(y, ref) <= TOL64


@pytest.mark.parametrize("p", [2, 4, 7])
def test_apply_assemble_f64(cw, orc, p):
    mesh = mesh_for(p)
    x = orc.gather(mesh, p, synth.global_vector(mesh, p, seed=20 + p))
    ref = orc.dss(mesh, p, orc.apply_local(mesh, p, 3, x))
    y = run_apply(cw, mesh, p, 3, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, x, assemble=True)
    assert rel_err(y, ref) <= TOL64


@pytest.mark.parametrize("prec", [0, 1, 2, 4], ids=["df64", "f64native", "f32", "bf16"])
@pytest.mark.parametrize("dims", [(4, 3, 5), (1, 3, 2), (2, 1, 1), (5, 1, 3), (9, 2, 2)])
@pytest.mark.parametrize("p", [1, 2, 4, 7])
@pytest.mark.parametrize("geom", [1, 2], ids=["stored", "recompute"])
def test_assemble_fused_x_matches_axis_passes(cw, p, dims, prec, geom):
    """The assembled apply sums the x-interfaces inside each operator tile in the kernel's epilogue
    and leaves the rest to the DSS: bit-identical to a local apply followed by the three axis passes
    of Algorithm struct_dss, for every tile size and staging mode (tiles that straddle x-rows and a
    ragged last tile included)."""
    import torch
    mesh = synth.box_mesh(*dims, perturb=0.1)
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, p, 3, geom, prec)
    x = torch.from_numpy(synth.cellwise_random(mesh, p, seed=40 + p)).cuda().to(op.vec_dtype)
    _, _, choices = op.variant()  # the default tile and the alternative (half of it)
    variants = [(0, 0)] if prec == 1 else [(c, st) for c in choices for st in (0, 1, 2)]
    if geom == 2 and prec != 1:  # recomputed geometry: default tile only
        variants = [(choices[0], st) for st in (0, 1, 2)]
    for cpb, stage in variants:
        if cpb:
            op.set_variant(cpb, stage)
        y_fused = op.apply(x, assemble=True)
        y_passes = op.dss(op.apply(x))
        torch.cuda.synchronize()
        assert torch.equal(y_fused, y_passes), (cpb, stage)


@pytest.mark.parametrize("prec,tol", [(2, 2e-6), (3, 1e-2), (4, 3e-2)], ids=["f32", "f32_bf16g", "bf16"])
@pytest.mark.parametrize("p", [1, 2, 4, 7])
def test_apply_reduced_precision_error(cw, orc, p, prec, tol):
    """Reduced precision has no parity bar from the paper; its error against the FP64 oracle is
    measured and bounded by what the storage precision allows."""
    mesh = mesh_for(p)
    x = orc.gather(mesh, p, synth.global_vector(mesh, p, seed=p))
    ref = orc.apply_local(mesh, p, 1, x)
    y = run_apply(cw, mesh, p, 1, cw.CW_GEOM_METRIC, prec, x)
    err = rel_err(y, ref)
    print(f"p={p} prec={prec} rel err {err:.3e}")
    assert err <= tol


@pytest.mark.parametrize("p", [1, 3, 6])
def test_gather_exact(cw, orc, p):
    import torch
    mesh = synth.box_mesh(4, 3, 2, perturb=0.1)
    ug = synth.global_vector(mesh, p, seed=3)
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, p, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64)
    x = op.gather(torch.from_numpy(ug).cuda())
    assert np.array_equal(to_np(x), orc.gather(mesh, p, ug))


@pytest.mark.parametrize("average", [False, True])
@pytest.mark.parametrize("dims", [(4, 3, 5), (1, 3, 2), (2, 1, 1)])
@pytest.mark.parametrize("p", [1, 2, 5])
def test_dss(cw, orc, p, dims, average):
    import torch
    mesh = synth.box_mesh(*dims)
    r = synth.cellwise_random(mesh, p, seed=5)
    ref = orc.dss(mesh, p, r)
    if average:
        kappa = orc.dss(mesh, p, np.ones_like(r))
        ref = ref / kappa
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, p, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64)
    v = torch.from_numpy(r).cuda()
    op.dss(v, average=average)
    torch.cuda.synchronize()
    assert rel_err(to_np(v), ref) <= 1e-15


@pytest.mark.parametrize("kind", [1, 3])
@pytest.mark.parametrize("p", [1, 3, 5])
def test_diagonal(cw, orc, p, kind):
    mesh = synth.box_mesh(3, 2, 3, perturb=0.2)
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, p, kind, cw.CW_GEOM_METRIC, cw.CW_PREC_F64)
    d = to_np(op.diagonal())
    ref = orc.gather(mesh, p, orc.diagonal(mesh, p, kind))
    assert rel_err(d, ref) <= TOL64


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("p", [1, 4])
def test_load_vector(cw, orc, p, which):
    mesh = synth.box_mesh(3, 3, 2, perturb=0.2)
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, p, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64)
    b = to_np(op.load_vector(which))
    assert rel_err(b, orc.load_vector(mesh, p, which)) <= TOL64


@pytest.mark.parametrize("prec", [0, 2, 4], ids=["df64", "f32", "bf16"])
@pytest.mark.parametrize("p", [1, 3, 4, 7])
def test_apply_all_variants(cw, orc, p, prec):
    """Every kernel variant (two tile sizes x direct loads, TMA staging, or TMA + L2 prefetch) gives
    the oracle's result;
    the mesh has a ragged last tile for both tile sizes."""
    import torch
    mesh = synth.box_mesh(3, 3, 5, perturb=0.2) if p < 7 else synth.box_mesh(3, 1, 3, perturb=0.2)
    x = orc.gather(mesh, p, synth.global_vector(mesh, p, seed=40 + p))
    ref = orc.apply_local(mesh, p, 3, x)
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, p, 3, cw.CW_GEOM_METRIC, prec)
    _, _, choices = op.variant()
    xd = torch.from_numpy(x).cuda().to(op.vec_dtype)
    tol = {0: TOL64, 2: 2e-6, 4: 3e-2}[prec]
    for cpb in choices:
        for stage in (0, 1, 2):
            op.set_variant(cpb, stage)
            y = op.apply(xd)
            torch.cuda.synchronize()
            assert rel_err(to_np(y), ref) <= tol, (cpb, stage)


def test_autotune_keeps_a_valid_variant(cw, orc):
    import torch
    p = 4
    mesh = synth.box_mesh(8, perturb=0.1)
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, p, 3, cw.CW_GEOM_METRIC, cw.CW_PREC_F64)
    x = op.gather(torch.from_numpy(synth.global_vector(mesh, p, seed=1)).cuda())
    y = op.empty()
    ms = op.autotune(x, y, reps=2)
    cpb, stage, choices = op.variant()
    assert ms > 0 and cpb in choices and stage in (0, 1, 2)
    y2 = op.apply(x)
    ref = orc.apply_local(mesh, p, 3, to_np(x))
    assert rel_err(to_np(y2), ref) <= TOL64


@pytest.mark.parametrize("nz", [1, 19, 40])
@pytest.mark.parametrize("geom", [1, 2], ids=["stored", "recompute"])
@pytest.mark.parametrize("assemble", [False, True])
@pytest.mark.parametrize("prec", [0, 2], ids=["df64", "f32"])
def test_apply_host_buffers(cw, orc, prec, assemble, geom, nz):
    """cw_apply_host (host input and output, chunked and pipelined) equals cw_apply on device data.
    z-slabs by layer count: 1 -> one slab; 19 -> 1, 2 x 8, 1, 1 (nominal 2 layers, ramp 1); 40 -> 1, 2,
    3 x 11, 1, 2, 1 (nominal 3, ramp 1, 2; a ragged middle slab)."""
    import torch
    p = 3
    mesh = synth.box_mesh(5, 4, nz, perturb=0.2)
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, p, 3, geom, prec)
    x = op.gather(torch.from_numpy(synth.global_vector(mesh, p, seed=3)).cuda())
    ref = op.apply(x, assemble=assemble)
    xh = x.cpu().pin_memory()
    yh = torch.full_like(xh, float("nan")).pin_memory()
    for _ in range(2):
        cw.cw_apply_host(op.handle, xh, yh, cw.CW_APPLY_ASSEMBLE if assemble else cw.CW_APPLY_LOCAL)
        torch.cuda.synchronize()
        assert torch.equal(yh, ref.cpu())


def test_create_reports_device_oom(cw):
    """An operator whose metric cannot fit in device memory (p=7, K+M, 240^3 cells: 396 GB of
    FP64 metric) fails with CW_ERR_OOM from cw_op_create, and the library stays usable."""
    mesh = synth.box_mesh(240)
    M = cw.Mesh.from_synth(mesh)
    with pytest.raises(cw.CwError) as ei:
        cw.Operator(M, 7, cw.CW_LAPLACE_MASS, cw.CW_GEOM_METRIC, cw.CW_PREC_F64)
    assert ei.value.status == cw.CW_ERR_OOM
    small = synth.box_mesh(2, 2, 2, perturb=0.1)
    op = cw.Operator(cw.Mesh.from_synth(small), 2, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64)
    assert op.L == 8 * 27


@pytest.mark.parametrize("perturb,freq,direction", [(0.1, None, None), (0.2, (2, 1, 3), (0.3, -1.0, 0.5)),
                                                    (0.0, None, None)])
def test_box_mesh_from_the_library(cw, orc, perturb, freq, direction):
    """cw_mesh_create_box builds the same deformed cube as the input generator: the operator on it
    matches the oracle on the generator's mesh."""
    p = 3
    kw = {} if freq is None else {"freq": freq, "direction": direction}
    mesh = synth.box_mesh(4, 3, 5, perturb=perturb, **kw)
    x = orc.gather(mesh, p, synth.global_vector(mesh, p, seed=7))
    ref = orc.apply_local(mesh, p, 3, x)
    import torch
    M = cw.Mesh.box(4, 3, 5, perturb=perturb, freq=freq, direction=direction)
    geom = cw.CW_GEOM_AFFINE if perturb == 0.0 else cw.CW_GEOM_METRIC
    op = cw.Operator(M, p, 3, geom, cw.CW_PREC_F64)
    y = to_np(op.apply(torch.from_numpy(x).cuda()))
    assert rel_err(y, ref) <= TOL64


@pytest.mark.parametrize("scale_exp,prec", [(-70, 0), (90, 0), (-600, 1), (600, 1)],
                         ids=["df64_2^-70", "df64_2^90", "f64native_2^-600", "f64native_2^600"])
def test_apply_inputs_far_from_unit_scale(cw, orc, scale_exp, prec):
    """Inputs scaled by a power of two (the exact output scales with them): the double-float operator
    keeps its accuracy while its intermediate values (the inputs times metric entries that scale like
    h and h^3, about 2^-11 at the smallest here) keep float pairs with a normal low part (above about
    2^-100; at an input scale of 2^-90 the error grew to 1e-11); the IEEE FP64 operator over the whole
    double range."""
    p, kind = 3, 3
    mesh = mesh_for(p)
    x = orc.gather(mesh, p, synth.global_vector(mesh, p, seed=9))
    ref = orc.apply_local(mesh, p, kind, x)
    s = 2.0 ** scale_exp
    y = run_apply(cw, mesh, p, kind, cw.CW_GEOM_METRIC, prec, x * s)
    assert rel_err(y / s, ref) <= TOL64
