"""Parity at the full workload sizes, in the launch configuration the benchmark times (autotuned
variants): the GPU output on a seeded sample of cells is compared with the oracle computed cell by
cell. Assembled outputs are checked on sampled cells through the oracle's apply on the 3x3x3
neighbourhood of each sampled cell followed by the oracle's global-index DSS restricted to it."""
import numpy as np
import pytest

import synth
from gpu_util import rel_err, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SWEEP_N = {1: 256, 2: 171, 3: 128, 4: 102, 5: 85, 6: 73, 7: 64}


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


def sample_cells(mesh, k, seed=0):
    rng = np.random.default_rng(seed)
    cells = rng.choice(mesh.ncells, k, replace=False)
    # always include the corners and a ragged-tail cell
    extra = np.array([0, mesh.nx - 1, mesh.ncells - 1, mesh.ncells - mesh.nx])
    return np.unique(np.concatenate([cells, extra]))


def cellwise_global_input(cw, orc, mesh, p, op, seed):
    import torch
    ug = synth.global_vector(mesh, p, seed=seed)
    x = op.gather(torch.from_numpy(ug).cuda())
    return ug, x


def oracle_local_on_cells(orc, mesh, p, kind, ug, cells):
    """Oracle LOCAL apply on the listed cells, input gathered from the global vector."""
    n3 = (p + 1) ** 3
    gidx = orc.global_index(mesh, p).reshape(mesh.ncells, n3)
    x = np.zeros(mesh.ncells * n3)
    xr = x.reshape(mesh.ncells, n3)
    xr[cells] = ug[gidx[cells]]
    return orc.apply_local(mesh, p, kind, x, cells)


def test_config2_q4_km_64cubed_local_and_assembled(cw, orc):
    """Config 2: Laplace + mass, Q4, 64^3 curved cells, FP64 (double-float), autotuned variant."""
    import torch
    p, kind = 4, 3
    mesh = synth.box_mesh(64, perturb=0.1)
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, p, kind, cw.CW_GEOM_METRIC, cw.CW_PREC_F64)
    ug, x = cellwise_global_input(cw, orc, mesh, p, op, seed=0)
    y = op.empty()
    op.autotune(x, y, reps=2)
    y = op.apply(x)
    ya = op.apply(x, assemble=True)
    torch.cuda.synchronize()
    n3 = (p + 1) ** 3
    cells = sample_cells(mesh, 48)
    ref = oracle_local_on_cells(orc, mesh, p, kind, ug, cells)
    got = to_np(y).reshape(mesh.ncells, n3)[cells]
    assert rel_err(got, ref) <= 1e-12
    # assembled: each sampled cell's copies = sum over the cells sharing each DoF (3x3x3 block)
    gidx = orc.global_index(mesh, p).reshape(mesh.ncells, n3)
    for c in cells[:12]:
        cx, cy, cz = c % 64, (c // 64) % 64, c // 4096
        nb = [(cx + a) + 64 * ((cy + b) + 64 * (cz + d)) for d in (-1, 0, 1) for b in (-1, 0, 1) for a in (-1, 0, 1)
              if 0 <= cx + a < 64 and 0 <= cy + b < 64 and 0 <= cz + d < 64]
        nb = np.array(sorted(nb))
        yl = oracle_local_on_cells(orc, mesh, p, kind, ug, nb)
        acc = {}
        for row, cc in zip(yl, nb):
            for loc, g in enumerate(gidx[cc]):
                acc[g] = acc.get(g, 0.0) + row[loc]
        ref_a = np.array([acc[g] for g in gidx[c]])
        assert rel_err(to_np(ya).reshape(mesh.ncells, n3)[c], ref_a) <= 1e-12


@pytest.mark.parametrize("p", range(1, 8))
def test_config3_degree_sweep(cw, orc, p):
    """Config 3: Laplace, ~2^27 cell-wise values, curved; FP64 at 1e-12, FP32 / BF16 error reported."""
    import torch
    N = SWEEP_N[p]
    mesh = synth.box_mesh(N, perturb=0.1)
    M = cw.Mesh.from_synth(mesh)
    n3 = (p + 1) ** 3
    cells = sample_cells(mesh, 24 if p < 6 else 8, seed=p)
    ug = synth.global_vector(mesh, p, seed=p)
    ref = oracle_local_on_cells(orc, mesh, p, 1, ug, cells)
    errs = {}
    for prec, tol in ((cw.CW_PREC_F64, 1e-12), (cw.CW_PREC_F32, 5e-6), (cw.CW_PREC_BF16, 5e-2)):
        op = cw.Operator(M, p, 1, cw.CW_GEOM_METRIC, prec)
        x = op.gather(torch.from_numpy(ug).cuda())
        y = op.empty()
        op.autotune(x, y, reps=1)
        y = op.apply(x)
        torch.cuda.synchronize()
        errs[prec] = rel_err(to_np(y).reshape(mesh.ncells, n3)[cells], ref)
        assert errs[prec] <= tol, (prec, errs[prec])
        del x, y
        op.close()
    print(f"p={p}: rel err f64 {errs[0]:.2e} f32 {errs[2]:.2e} bf16 {errs[4]:.2e}")


def test_config4_poisson_q3_128cubed(cw, orc):
    """Config 4: the IR-FP32 solve reaches 1e-10 (native-FP64 residual) and its discretisation error
    matches the FP64 solve's."""
    import torch
    p = 3
    mesh = synth.box_mesh(128, perturb=0.1)
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, p, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
    b = op.load_vector(0)
    u1, s1, rc1 = op.cg_solve(b, rtol=1e-10, maxit=20000, mode=cw.CW_CG_IR_F32)
    assert s1.rel_residual <= 1e-10
    u0, s0, rc0 = op.cg_solve(b, rtol=1e-10, maxit=20000, mode=cw.CW_CG_F64)
    assert s0.rel_residual <= 1e-10
    assert rel_err(to_np(u1), to_np(u0)) <= 1e-8
    # the load vector on sampled cells against the oracle
    cells = sample_cells(mesh, 32)
    n3 = (p + 1) ** 3
    bref = orc.load_vector(synth.box_mesh(128, perturb=0.1), p).reshape(mesh.ncells, n3)[cells]
    assert rel_err(to_np(b).reshape(mesh.ncells, n3)[cells], bref) <= 1e-12


def test_config5_batched(cw, orc):
    """Config 5: 16 RHS on Q5 64^3 + 48 uneven problems in one graph launch (grouped mode, autotuned):
    sampled cells of every right-hand side of the big problem and of 8 small problems."""
    import torch
    probs = synth.batched_problem_list(48, seed=0)
    ops, xs, ys, nrhs, meshes, ugs = [], [], [], [], [], []
    big = synth.box_mesh(64, perturb=0.1)
    Mb = cw.Mesh.from_synth(big)
    opb = cw.Operator(Mb, 5, 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64)
    xb = torch.empty((16, opb.L), dtype=torch.float64, device="cuda")
    ugb = [synth.global_vector(big, 5, seed=r) for r in range(16)]
    for r in range(16):
        opb.gather(torch.from_numpy(ugb[r]).cuda(), xb[r])
    ops.append(opb); xs.append(xb); ys.append(torch.empty_like(xb)); nrhs.append(16); meshes.append((big, Mb)); ugs.append(ugb)
    for pr in probs:
        m = synth.box_mesh(pr["n"], perturb=0.1, freq=pr["freq"], direction=pr["direction"])
        Mm = cw.Mesh.from_synth(m)
        o = cw.Operator(Mm, pr["p"], 1, cw.CW_GEOM_METRIC, cw.CW_PREC_F64)
        ug = synth.global_vector(m, pr["p"], seed=pr["seed"])
        x = o.gather(torch.from_numpy(ug).cuda()).view(1, -1)
        ops.append(o); xs.append(x); ys.append(torch.empty_like(x)); nrhs.append(1); meshes.append((m, Mm)); ugs.append([ug])
    B = cw.Batch(ops, nrhs, xs, ys)
    B.autotune(reps=1)
    B.launch(graph=True)
    torch.cuda.synchronize()
    checks = [0] + list(range(1, 49, 6))
    for i in checks:
        (m, _), o, y, R = meshes[i], ops[i], ys[i], nrhs[i]
        p = o.degree
        n3 = (p + 1) ** 3
        cells = sample_cells(m, 6, seed=i)
        for r in (range(0, 16, 5) if R > 1 else [0]):
            ref = oracle_local_on_cells(orc, m, p, 1, ugs[i][r], cells)
            assert rel_err(to_np(y[r]).reshape(m.ncells, n3)[cells], ref) <= 1e-12, (i, r)
    B.close()


def test_apply_past_2e31_cellwise_values(cw, orc):
    """162^3 cells at p = 7 hold 2,176,782,336 cell-wise values, more than 2^31: the LOCAL and the
    assembled apply (FP32, mass) on cells at both ends of the vector and on both sides of value 2^31,
    each against the oracle on the cell's 3x3x3 neighbourhood cut from the same mesh (the local output
    of a cell depends on its own vertices and values only; every cell sharing one of its DoFs is in the
    neighbourhood, so the oracle's DSS there gives its assembled values)."""
    import torch
    p, kind, n = 7, 2, 162
    n3 = (p + 1) ** 3
    mesh = synth.box_mesh(n, perturb=0.1)
    op = cw.Operator(cw.Mesh.from_synth(mesh), p, kind, cw.CW_GEOM_METRIC, cw.CW_PREC_F32)
    assert op.L == n ** 3 * n3 and op.L > 2 ** 31
    gen = torch.Generator(device="cuda")
    gen.manual_seed(31)
    x = torch.rand(op.L, dtype=torch.float32, device="cuda", generator=gen).sub_(0.5)
    y = op.apply(x)
    ya = op.apply(x, assemble=True)
    torch.cuda.synchronize()
    straddle = 2 ** 31 // n3  # the cell whose values reach past 2^31
    rng = np.random.default_rng(7)
    cells = sorted({0, n - 1, straddle - 1, straddle, straddle + 1, n ** 3 - n * n + 5 * n + 7, n ** 3 - 1,
                    *rng.integers(straddle, n ** 3, 4).tolist()})
    for c in cells:
        cx, cy, cz = c % n, (c // n) % n, c // (n * n)
        x0, x1 = max(cx - 1, 0), min(cx + 2, n)
        y0, y1 = max(cy - 1, 0), min(cy + 2, n)
        z0, z1 = max(cz - 1, 0), min(cz + 2, n)
        sub = synth.Mesh(x1 - x0, y1 - y0, z1 - z0,
                         np.ascontiguousarray(mesh.verts[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1]), False)
        ids = np.array([(i + x0) + n * ((j + y0) + n * (k + z0))
                        for k in range(z1 - z0) for j in range(y1 - y0) for i in range(x1 - x0)], dtype=np.int64)
        idx = torch.from_numpy((ids[:, None] * n3 + np.arange(n3)[None, :]).ravel()).cuda()
        xs = to_np(x.index_select(0, idx)).astype(np.float64)
        yl = orc.apply_local(sub, p, kind, xs).reshape(len(ids), n3)
        ys = orc.dss(sub, p, yl.ravel()).reshape(len(ids), n3)
        kc = int(np.nonzero(ids == c)[0][0])
        got = to_np(y[c * n3:(c + 1) * n3]).astype(np.float64)
        got_a = to_np(ya[c * n3:(c + 1) * n3]).astype(np.float64)
        assert rel_err(got, yl[kc]) <= 5e-6, c
        assert rel_err(got_a, ys[kc]) <= 5e-6, c
