"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only draws random numbers and lays out mesh vertex coordinates; it holds none of the
finite-element arithmetic (no basis functions, quadrature, gather/scatter or operator). Both the
CPU oracle and the CUDA library receive exactly these arrays.

Inputs (the paper's cube / ball sweeps are not available, so these stand in for them):
  * a box mesh of the unit cube with ``nx*ny*nz`` hexahedra, vertex ``(ix, iy, iz)`` at
    ``(ix/nx, iy/ny, iz/nz)`` optionally moved by a smooth sinusoidal displacement of amplitude
    ``0.1*h`` that vanishes on the boundary of the cube (so the domain stays the unit cube);
  * global vectors of length ``(nx*p+1)*(ny*p+1)*(nz*p+1)`` drawn uniform in [-1, 1];
  * raw cell-wise arrays of length ``E*(p+1)^3`` drawn uniform in [-1, 1] (unassembled duals);
  * multi-block meshes (several structured blocks glued face to face with seeded relative
    orientations): the unit cube cut into nb^3 blocks, and the 7-block "cube in cube" (an inner cube
    and six frustum-shaped shell blocks, edges shared by three blocks, vertices by four), the stand-in
    for the paper's curved multi-block ball.
"""
from dataclasses import dataclass
import math
import numpy as np

__all__ = ["Mesh", "box_mesh", "refine", "global_vector", "cellwise_random", "batched_problem_list",
           "global_len", "cellwise_len", "MultiBlock", "cube_blocks", "cube_in_cube", "rotate_block"]


@dataclass
class Mesh:
    nx: int
    ny: int
    nz: int
    verts: np.ndarray  # float64, shape (nz+1, ny+1, nx+1, 3), C-contiguous
    affine: bool       # True when no displacement was applied (uniform Cartesian cells)

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz


def box_mesh(nx, ny=None, nz=None, perturb=0.0, freq=(1, 1, 1), direction=None) -> Mesh:
    """Unit-cube box mesh; ``perturb`` is the displacement amplitude in units of h = 1/max(n).

    Displacement: ``perturb*h * sin(2 pi fx X) sin(2 pi fy Y) sin(2 pi fz Z) * direction`` with
    ``direction`` a unit vector (default (1,1,1)/sqrt(3)). It is zero on the boundary faces.
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    x = np.arange(nx + 1, dtype=np.float64) / nx
    y = np.arange(ny + 1, dtype=np.float64) / ny
    z = np.arange(nz + 1, dtype=np.float64) / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    verts = np.stack([X, Y, Z], axis=-1)
    if perturb != 0.0:
        h = 1.0 / max(nx, ny, nz)
        d = np.ones(3) / math.sqrt(3.0) if direction is None else np.asarray(direction, np.float64)
        d = d / np.linalg.norm(d)
        s = (np.sin(2 * np.pi * freq[0] * X) * np.sin(2 * np.pi * freq[1] * Y)
             * np.sin(2 * np.pi * freq[2] * Z))
        verts = verts + perturb * h * s[..., None] * d[None, None, None, :]
        # snap the boundary exactly (sin(2 pi k) is not exactly 0 in floating point)
        verts[:, :, 0, 0] = 0.0
        verts[:, :, -1, 0] = 1.0
        verts[:, 0, :, 1] = 0.0
        verts[:, -1, :, 1] = 1.0
        verts[0, :, :, 2] = 0.0
        verts[-1, :, :, 2] = 1.0
    return Mesh(nx, ny, nz, np.ascontiguousarray(verts), affine=(perturb == 0.0))


def refine(mesh: Mesh) -> Mesh:
    """The next level of a uniform mesh hierarchy: every cell split into 2 x 2 x 2 children by its
    own trilinear map (Sec. 3: nested meshes, each cell of a level obtained by refining a cell of
    the previous one). Child vertices are the parent map at the half points, i.e. along every axis
    the old vertex rows are kept and the midpoint of each pair of neighbours is inserted; the
    children are trilinear images again, so the finite-element spaces of the levels are nested."""
    v = mesh.verts
    for axis in (2, 1, 0):  # x, y, z vertex index (array axes 2, 1, 0)
        n = v.shape[axis]
        shape = list(v.shape)
        shape[axis] = 2 * n - 1
        w = np.empty(shape)
        even = [slice(None)] * 4
        odd = [slice(None)] * 4
        even[axis] = slice(0, None, 2)
        odd[axis] = slice(1, None, 2)
        lo = [slice(None)] * 4
        hi = [slice(None)] * 4
        lo[axis] = slice(0, n - 1)
        hi[axis] = slice(1, n)
        w[tuple(even)] = v
        w[tuple(odd)] = 0.5 * (v[tuple(lo)] + v[tuple(hi)])
        v = w
    return Mesh(2 * mesh.nx, 2 * mesh.ny, 2 * mesh.nz, np.ascontiguousarray(v), affine=mesh.affine)


def global_len(mesh: Mesh, p: int) -> int:
    return (mesh.nx * p + 1) * (mesh.ny * p + 1) * (mesh.nz * p + 1)


def cellwise_len(mesh: Mesh, p: int) -> int:
    return mesh.ncells * (p + 1) ** 3


def global_vector(mesh: Mesh, p: int, seed: int = 0) -> np.ndarray:
    """Uniform[-1,1] global vector in global lexicographic order (x fastest)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, global_len(mesh, p))


def cellwise_random(mesh: Mesh, p: int, seed: int = 0) -> np.ndarray:
    """Uniform[-1,1] raw cell-wise array (no continuity), layout [cell][k][j][i]."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, cellwise_len(mesh, p))


def batched_problem_list(count: int = 48, seed: int = 0, lo: int = 8, hi: int = 48,
                         degrees=(2, 3, 5, 7)):
    """Uneven batch: problem i has N_i ~ U{lo..hi} cells per direction, degree degrees[i % 4],
    a displacement with seeded integer frequencies in {1,2,3} and a seeded unit direction."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(lo, hi + 1))
        r = np.random.default_rng(i)
        freq = tuple(int(f) for f in r.integers(1, 4, 3))
        d = r.normal(size=3)
        out.append(dict(n=n, p=degrees[i % len(degrees)], freq=freq, direction=d / np.linalg.norm(d),
                        seed=i))
    return out


# ----------------------------------------------------------------------------- multi-block
@dataclass
class MultiBlock:
    blocks: list       # list of Mesh, each a structured block with its own local axes
    lo: float          # the domain is the cube [lo, hi]^3 (its boundary carries the Dirichlet nodes)
    hi: float


def _proper_rotations():
    """The 24 orientation-preserving symmetries of the index cube as (axis permutation, flips): a
    permutation of odd parity needs an odd number of flips (so the trilinear maps keep det J > 0)."""
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        inv = sum(1 for i in range(3) for j in range(i + 1, 3) if perm[i] > perm[j]) % 2
        for flips in itertools.product((0, 1), repeat=3):
            if (inv + sum(flips)) % 2 == 0:
                out.append((perm, flips))
    return out


def rotate_block(mesh: Mesh, rot) -> Mesh:
    """The same cells with the block's local index axes permuted and reversed by a proper rotation
    ``rot = (perm, flips)``: local axis a of the result runs along old axis perm[a], reversed when
    flips[a] (the physical cells are unchanged, only their local numbering)."""
    perm, flips = rot
    v = mesh.verts  # array axes (z, y, x, 3)
    n_old = (mesh.nx, mesh.ny, mesh.nz)
    # new local axis a (0 = x) comes from old local axis perm[a]; array axis of local axis a is 2 - a
    w = np.transpose(v, (2 - perm[2], 2 - perm[1], 2 - perm[0], 3))
    for a in range(3):
        if flips[a]:
            w = np.flip(w, axis=2 - a)
    n = tuple(n_old[perm[a]] for a in range(3))
    return Mesh(n[0], n[1], n[2], np.ascontiguousarray(w), affine=mesh.affine)


def cube_blocks(nb=2, ncell=2, perturb=0.0, seed=0, rotate=True) -> MultiBlock:
    """The unit cube cut into nb^3 cubic blocks of ncell^3 cells: the cells of box_mesh(nb*ncell,
    perturb) exactly, each block with a seeded proper rotation of its local axes (so neighbouring
    blocks meet in every relative orientation)."""
    g = box_mesh(nb * ncell, perturb=perturb)
    rots = _proper_rotations()
    rng = np.random.default_rng(seed)
    blocks = []
    for bz in range(nb):
        for by in range(nb):
            for bx in range(nb):
                sub = g.verts[bz * ncell:(bz + 1) * ncell + 1, by * ncell:(by + 1) * ncell + 1,
                              bx * ncell:(bx + 1) * ncell + 1]
                m = Mesh(ncell, ncell, ncell, np.ascontiguousarray(sub), affine=g.affine)
                blocks.append(rotate_block(m, rots[int(rng.integers(len(rots)))]) if rotate else m)
    return MultiBlock(blocks, 0.0, 1.0)


def cube_in_cube(ncell=2, a=0.5, b=1.0, seed=0, rotate=True) -> MultiBlock:
    """Seven blocks of ncell^3 cells filling [-b, b]^3: the inner cube [-a, a]^3 and, on each of its
    faces, a shell block whose cells run from the inner face out to the outer face along the rays
    from the origin (point r(t) F(u, v) with F on the unit cube's face, r from a to b). The shell
    cells are trilinear but not affine. Edges of the inner cube are shared by three blocks, its
    corners by four. With ``rotate`` every block gets a seeded proper rotation of its local axes."""
    s = np.linspace(-1.0, 1.0, ncell + 1)
    t = np.linspace(0.0, 1.0, ncell + 1)
    K, J, I = np.meshgrid(s, s, s, indexing="ij")
    blocks = [Mesh(ncell, ncell, ncell, np.ascontiguousarray(a * np.stack([I, J, K], axis=-1)), affine=True)]
    for axis in range(3):
        beta, gamma = (axis + 1) % 3, (axis + 2) % 3
        for sign in (1.0, -1.0):
            # local axes (i, j, k) = (u, v, radial); for the negative face u and v swap to keep det J > 0
            Kt, Jv, Iu = np.meshgrid(t, s, s, indexing="ij")
            if sign < 0:
                Iu, Jv = Jv, Iu
            F = np.zeros(Kt.shape + (3,))
            F[..., axis] = sign
            F[..., beta] = Iu
            F[..., gamma] = Jv
            r = (1.0 - Kt) * a + Kt * b
            blocks.append(Mesh(ncell, ncell, ncell, np.ascontiguousarray(r[..., None] * F), affine=False))
    if rotate:
        rots = _proper_rotations()
        rng = np.random.default_rng(seed)
        blocks = [rotate_block(m, rots[int(rng.integers(len(rots)))]) for m in blocks]
    return MultiBlock(blocks, -b, b)
