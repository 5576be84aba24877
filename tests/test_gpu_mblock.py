"""Multi-block meshes on the GPU (Sec. 4.3, Algorithm unstruct_dss) against the oracle's multi-block
numbering (oracle.mblock, by node position): the library's numbering (block-vertex identities and
canonical edge and face frames) must be the same partition of the cell-wise entries, its DSS the
oracle's S, its assembled apply and diagonal the oracle's, and its solve the oracle's direct solve."""
import numpy as np
import pytest

import synth
from gpu_util import rel_err, to_np

pytestmark = pytest.mark.gpu


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


@pytest.fixture(scope="module")
def omb(orc):
    from oracle import mblock
    return mblock


MESHES = {
    "cube_2x2x2_rotated": lambda: synth.cube_blocks(2, 2, perturb=0.1, seed=5),
    "cube_3x3x3_rotated": lambda: synth.cube_blocks(3, 1, perturb=0.0, seed=7),
    "cube_in_cube_n1": lambda: synth.cube_in_cube(1, seed=2),
    "cube_in_cube_n3": lambda: synth.cube_in_cube(3, seed=4),
}


def build(cw, mbm, p, kind=1, prec=0, bc=1):
    Ms = [cw.Mesh.from_synth(m) for m in mbm.blocks]
    ops = [cw.Operator(M, p, kind, cw.CW_GEOM_METRIC, prec, bc) for M in Ms]
    return Ms, ops, cw.MultiBlock(ops)


def dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_numbering_and_dss_match_oracle(cw, orc, omb, name, p):
    import torch
    mbm = MESHES[name]()
    ref = omb.MultiBlockMesh(mbm, p)
    Ms, ops, mb = build(cw, mbm, p)
    assert mb.L == ref.L and mb.NG == ref.NG
    g = mb.global_index()
    # the same partition of the entries into DoFs: a bijection between the two numberings
    pairs = np.unique(np.stack([g, ref.gidx], axis=1), axis=0)
    assert len(pairs) == ref.NG and len(np.unique(pairs[:, 0])) == ref.NG
    x = np.random.default_rng(p).uniform(-1.0, 1.0, ref.L)  # raw cell-wise values, no continuity
    for average in (False, True):
        v = dev(x, torch.float64)
        mb.dss(v, average=average)
        want = ref.dss(x) / (ref.valence() if average else 1.0)
        assert rel_err(to_np(v), want) <= 1e-14, average


@pytest.mark.parametrize("name", ["cube_2x2x2_rotated", "cube_in_cube_n3"])
@pytest.mark.parametrize("kind", [1, 3])
@pytest.mark.parametrize("p", [2, 3])
def test_assembled_apply_and_diagonal_match_oracle(cw, orc, omb, name, p, kind):
    import torch
    mbm = MESHES[name]()
    ref = omb.MultiBlockMesh(mbm, p)
    Ms, ops, mb = build(cw, mbm, p, kind)
    ug = np.random.default_rng(p + kind).uniform(-1, 1, ref.NG)
    x = ref.gather(ug)
    y = to_np(mb.apply(dev(x, torch.float64), assemble=True))
    want = ref.dss(ref.apply_local(kind, x))
    assert rel_err(y, want) <= 1e-12
    A = ref.assemble(kind)
    assert rel_err(to_np(mb.diagonal()), ref.gather(A.diagonal())) <= 1e-12
    # the FP32 blocks through the same tables
    Ms32, ops32, mb32 = build(cw, mbm, p, kind, prec=cw.CW_PREC_F32)
    y32 = to_np(mb32.apply(dev(x, torch.float32), assemble=True))
    assert rel_err(y32, want) <= 2e-6


@pytest.mark.parametrize("name", ["cube_2x2x2_rotated", "cube_in_cube_n3"])
def test_solve_matches_oracle_direct_solve(cw, orc, omb, name):
    import torch
    p = 2
    mbm = MESHES[name]()
    ref = omb.MultiBlockMesh(mbm, p)
    Ms, ops, mb = build(cw, mbm, p)
    b = np.concatenate([orc.load_vector(m, p, orc.PROBLEM_SINE) for m in mbm.blocks])
    A = ref.assemble(1)
    ud = ref.gather(orc.direct_solve(A, ref.scatter_add(b), ref.boundary_mask()))
    u, st, rc = mb.cg_solve(dev(b, torch.float64), rtol=1e-12, maxit=5000)
    un = to_np(u)
    res = (np.linalg.norm(ref.boundary_mask() * (ref.scatter_add(b) - A @ (ref.scatter_add(un) / ref.scatter_add(np.ones_like(un)))))
           / np.linalg.norm(ref.boundary_mask() * ref.scatter_add(b)))
    print(f"{name}: {st.iterations} it, residual {st.rel_residual:.2e} (oracle {res:.2e}), error {rel_err(un, ud):.2e}")
    assert st.rel_residual <= 1e-12 and res <= 1e-10
    assert rel_err(un, ud) <= 1e-10


def test_shared_dof_sets_of_the_cube_in_cube(cw, omb):
    """Codimension sets of the 7-block mesh. ncell = 1, p = 1: only vertices, the 8 inner-cube corners
    (four blocks each) and the 8 outer corners (three shell blocks each). ncell = 2, p = 2 (5 x 5 nodes
    on a block face, 3 x 3 inside it, 3 inside a block edge): 18 glued block faces (6 around the inner
    cube, 12 between neighbouring shells); 32 shared block edges (12 inner-cube edges, 12 outer-cube
    edges, 8 radial edges from inner to outer corners); the same 16 vertices."""
    Ms, ops, mb = build(cw, synth.cube_in_cube(1, seed=0), 1)
    assert mb.shared_dofs() == (0, 0, 16)
    Ms, ops, mb = build(cw, synth.cube_in_cube(2, seed=0), 2)
    assert mb.shared_dofs() == (18 * 9, 32 * 3, 8 + 8)


def test_argument_errors(cw):
    mbm = synth.cube_in_cube(1, seed=0)
    Ms = [cw.Mesh.from_synth(m) for m in mbm.blocks]
    ops = [cw.Operator(M, 2 if i else 1, 1, cw.CW_GEOM_METRIC, 0, 1) for i, M in enumerate(Ms)]
    import ctypes
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 7)(*[o.handle.value for o in ops])
    assert cw.load().cw_mblock_create(arr, 7, ctypes.byref(h)) == cw.CW_ERR_ARG
    arr2 = (ctypes.c_void_p * 2)(ops[1].handle.value, ops[1].handle.value)
    assert cw.load().cw_mblock_create(arr2, 2, ctypes.byref(h)) == cw.CW_ERR_ARG
