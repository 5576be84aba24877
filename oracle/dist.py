"""Slab-partitioned cell-wise DSS and Jacobi-PCG over torch.distributed, FP64 (the exchange step of a
multi-GPU partition; Sec. 4.3 and Sec. 4.4).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: the CUDA library never imports or calls it.

Partition: rank r of W owns the whole cell layers cz in [z0_r, z1_r) (z0_r = r nz / W, rounded down).
Cells are numbered with z slowest, so a rank's part of a cell-wise vector is one contiguous slice of
the global vector, and its cells form the box sub-mesh of those layers.

DSS across ranks: every step of the cell-wise path is local except the direct stiffness summation
(Sec. 4.3). Algorithm struct_dss sums along x, then y, then z; with z-slabs the x and y passes and the
z interfaces inside a slab are the slab's own DSS, after which each face layer on a slab interface
already holds the sum over its side's copies (edges and corners included). One exchange per
interface then completes the z pass: each side sends its face layer (k = p of its top cell layer,
k = 0 of its bottom layer) and writes s = (lower layer) + (upper layer), the same two-operand sum on
both sides.

Jacobi-PCG: the cell-wise primal-dual iteration of Sec. 4.4 on the slabs; every inner product pairs
a raw dual with a continuous primal vector, so a local dot plus one sum over ranks (all_reduce) gives
the global value without assembly.
"""
import numpy as np

from . import all_element_matrices, apply_local, dss as local_dss


class Slab:
    """Rank ``rank``'s part of ``mesh``: cell layers [z0, z1) as a box sub-mesh."""

    def __init__(self, mesh, rank, world):
        if not 1 <= world <= mesh.nz:
            raise ValueError("need 1 <= world <= nz (whole cell layers per rank)")
        self.rank, self.world = rank, world
        self.z0 = rank * mesh.nz // world
        self.z1 = (rank + 1) * mesh.nz // world
        self.nx, self.ny, self.nz = mesh.nx, mesh.ny, self.z1 - self.z0
        self.verts = np.ascontiguousarray(mesh.verts[self.z0:self.z1 + 1])
        self.gnz = mesh.nz

    @property
    def ncells(self):
        return self.nx * self.ny * self.nz

    def part(self, v, p):
        """This rank's slice of a global cell-wise vector."""
        n3 = (p + 1) ** 3
        per_layer = self.nx * self.ny * n3
        return np.ascontiguousarray(v[self.z0 * per_layer:self.z1 * per_layer])


def _exchange(send_up, send_down, rank, world):
    """Send the top layer to rank+1 and the bottom layer to rank-1; return (from_up, from_down)."""
    import torch
    import torch.distributed as dist
    reqs, from_up, from_down = [], None, None
    if rank + 1 < world:
        from_up = torch.empty_like(send_up)
        reqs.append(dist.isend(send_up, rank + 1))
        reqs.append(dist.irecv(from_up, rank + 1))
    if rank > 0:
        from_down = torch.empty_like(send_down)
        reqs.append(dist.isend(send_down, rank - 1))
        reqs.append(dist.irecv(from_down, rank - 1))
    for r in reqs:
        r.wait()
    return from_up, from_down


def dss(slab, p, v):
    """S v on the whole mesh, computed as the slab's DSS plus one face-layer exchange per slab
    interface (this rank's part in, this rank's part out)."""
    import torch
    n = p + 1
    z = local_dss(slab, p, v).reshape(slab.nz, slab.ny, slab.nx, n, n, n)  # [cz][cy][cx][k][j][i]
    top = torch.from_numpy(np.ascontiguousarray(z[-1, :, :, p]))
    bottom = torch.from_numpy(np.ascontiguousarray(z[0, :, :, 0]))
    from_up, from_down = _exchange(top, bottom, slab.rank, slab.world)
    if from_up is not None:    # this rank's top layer is the lower side of the interface
        z[-1, :, :, p] = top.numpy() + from_up.numpy()
    if from_down is not None:  # this rank's bottom layer is the upper side
        z[0, :, :, 0] = from_down.numpy() + bottom.numpy()
    return z.reshape(-1)


def allsum(x):
    """Sum of a float over all ranks."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t)
    return float(t[0])


def dirichlet_mask(slab, p):
    """1 on copies of interior DoFs of the whole cube, 0 on copies of its boundary DoFs."""
    n = p + 1
    i = np.arange(n)
    cx = np.arange(slab.nx)[:, None]
    cy = np.arange(slab.ny)[:, None]
    cz = np.arange(slab.z0, slab.z1)[:, None]
    bx = ((cx == 0) & (i == 0)) | ((cx == slab.nx - 1) & (i == p))    # [cx][i]
    by = ((cy == 0) & (i == 0)) | ((cy == slab.ny - 1) & (i == p))    # [cy][j]
    bz = ((cz == 0) & (i == 0)) | ((cz == slab.gnz - 1) & (i == p))   # [cz][k]
    bnd = (bz[:, None, None, :, None, None] | by[None, :, None, None, :, None]
           | bx[None, None, :, None, None, :])
    return (~bnd).astype(np.float64).reshape(-1)


def inverse_diagonal(slab, p, kind):
    """Cell-wise masked inverse of diag(A_CG): element diagonals, summed across all copies by the
    distributed DSS, inverted, zero on the Dirichlet copies (Eq. (jacobi_recap))."""
    A = all_element_matrices(slab, p, kind)
    d = dss(slab, p, np.ascontiguousarray(np.diagonal(A, axis1=1, axis2=2)).reshape(-1))
    return dirichlet_mask(slab, p) / d


def pcg(slab, p, kind, b, iterations):
    """Jacobi-preconditioned CG, cell-wise primal-dual form, for a fixed number of iterations from
    u = 0; b is this rank's part of the raw dual right-hand side. Returns this rank's part of each
    iterate u_0 .. u_iterations."""
    dinv = inverse_diagonal(slab, p, kind)
    u = np.zeros_like(b)
    r = b.copy()
    z = dinv * dss(slab, p, r)
    d = z.copy()
    rho = allsum(r @ z)
    its = [u.copy()]
    for _ in range(iterations):
        q = apply_local(slab, p, kind, d)
        alpha = rho / allsum(d @ q)
        u = u + alpha * d
        r = r - alpha * q
        z = dinv * dss(slab, p, r)
        rho_new = allsum(r @ z)
        d = z + (rho_new / rho) * d
        rho = rho_new
        its.append(u.copy())
    return its
