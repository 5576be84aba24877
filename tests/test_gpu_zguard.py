"""Guard bands: each entry point writes exactly its output range. Outputs are views into larger
NaN-filled buffers with K sentinels on each side; after the call the sentinels are intact and the
whole output range was written. Odd mesh sizes give ragged tiles for every tile shape."""
import pytest

import synth

pytestmark = pytest.mark.gpu

K = 64  # sentinels per side: 512 bytes for FP64, so the views keep 16-byte alignment


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


def guarded(n, dtype):
    import torch
    full = torch.full((n + 2 * K,), float("nan"), dtype=dtype, device="cuda")
    return full, full[K:K + n]


def intact(full, n):
    import torch
    torch.cuda.synchronize()
    return bool(full[:K].isnan().all()) and bool(full[K + n:].isnan().all())


def mesh_for(p):
    return synth.box_mesh(3, 1, 5, perturb=0.2) if p < 7 else synth.box_mesh(3, 1, 3, perturb=0.2)


@pytest.mark.parametrize("p", [1, 4, 7])
@pytest.mark.parametrize("prec", [0, 2, 4], ids=["f64", "f32", "bf16"])
def test_apply_gather_dss_write_only_their_range(cw, p, prec):
    import torch
    mesh = mesh_for(p)
    M = cw.Mesh.from_synth(mesh)
    ug = torch.from_numpy(synth.global_vector(mesh, p, seed=1)).cuda()
    for geom in (cw.CW_GEOM_METRIC, cw.CW_GEOM_RECOMPUTE):
        op = cw.Operator(M, p, cw.CW_LAPLACE_MASS, geom, prec)
        xf, x = guarded(op.L, op.vec_dtype)
        op.gather(ug, x)
        assert intact(xf, op.L) and not x.isnan().any()
        _, _, choices = op.variant()
        variants = [(c, s) for c in choices for s in (0, 1, 2)] if geom == cw.CW_GEOM_METRIC else [(0, 0), (0, 2)]
        for cpb, stage in variants:
            op.set_variant(cpb, stage)
            for assemble in (False, True):
                yf, y = guarded(op.L, op.vec_dtype)
                op.apply(x, y, assemble=assemble)
                assert intact(yf, op.L) and not y.isnan().any(), (geom, cpb, stage, assemble)
        for average in (False, True):
            vf, v = guarded(op.L, op.vec_dtype)
            v.copy_(x)
            op.dss(v, average)
            assert intact(vf, op.L) and not v.isnan().any()
        op.close()


def test_diagonal_load_vector_and_solve_write_only_their_range(cw):
    import torch
    p = 3
    mesh = synth.box_mesh(3, 2, 5, perturb=0.2)
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, p, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
    df, d = guarded(op.L, torch.float64)
    cw.cw_diagonal(op.handle, d)
    assert intact(df, op.L) and not d.isnan().any()
    bf, b = guarded(op.L, torch.float64)
    cw.cw_load_vector(op.handle, 0, b)
    assert intact(bf, op.L) and not b.isnan().any()
    for mode in (cw.CW_CG_F64, cw.CW_CG_IR_F32):
        uf, u = guarded(op.L, torch.float64)
        op.cg_solve(b, u, rtol=1e-8, maxit=500, mode=mode)
        assert intact(uf, op.L) and intact(bf, op.L) and not u.isnan().any()


def test_batch_and_host_apply_write_only_their_range(cw):
    import torch
    ops, xs, ys, fulls, nrhs = [], [], [], [], []
    for i, (n, p, R) in enumerate(((3, 2, 2), (2, 5, 1), (3, 7, 1))):
        m = synth.box_mesh(n, n + 1, max(1, n - 1), perturb=0.15)
        op = cw.Operator(cw.Mesh.from_synth(m), p, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, cw.CW_PREC_F64)
        xf, x = guarded(R * op.L, torch.float64)
        x.copy_(torch.from_numpy(synth.cellwise_random(m, p, seed=i)).cuda().repeat(R))
        yf, y = guarded(R * op.L, torch.float64)
        ops.append(op)
        xs.append(x)
        ys.append(y)
        fulls.append(yf)
        nrhs.append(R)
    for mode in (cw.CW_BATCH_GROUPED, cw.CW_BATCH_SINGLE):
        B = cw.Batch(ops, nrhs, xs, ys)
        B.set_mode(mode)
        B.launch()
        for yf, y, o, R in zip(fulls, ys, ops, nrhs):
            assert intact(yf, R * o.L) and not y.isnan().any()
        B.close()
    # host-buffer apply: guard bands around the host output
    op = ops[0]
    xh = xs[0][:op.L].cpu().pin_memory()
    yh_full = torch.full((op.L + 2 * K,), float("nan"), dtype=torch.float64).pin_memory()
    yh = yh_full[K:K + op.L]
    for flags in (cw.CW_APPLY_LOCAL, cw.CW_APPLY_ASSEMBLE):
        cw.cw_apply_host(op.handle, xh, yh, flags)
        torch.cuda.synchronize()
        assert bool(yh_full[:K].isnan().all()) and bool(yh_full[K + op.L:].isnan().all())
        assert not yh.isnan().any()
