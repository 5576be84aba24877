"""Multi-block meshes in cell-wise storage, FP64 (Sec. 4.3, the unstructured inter-block interfaces).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: the CUDA library never imports or calls it.

A multi-block mesh is a list of structured blocks (each a box of trilinear cells with its own local
axes) glued face to face. Its cell-wise vector is the concatenation of the blocks' cell-wise vectors
(block after block, each in its own [cell][k][j][i] layout).

The global numbering is the plain definition: two cell-wise entries are copies of one global DoF when
their nodes sit at the same point of space. Node positions come from the oracle's own trilinear maps
(``node_coords``) and are matched after rounding to 1e-7 (nodes of the test meshes are at least ~1e-3
apart; copies agree to ~1e-15). Everything else follows from the index, as on a single block:
G by index, G^T by accumulation, S = G G^T, A_CG = sum over cells of P_K^T A_K P_K.
The GPU library finds the same coupling another way (block-vertex identities and the orientation of
each shared face and edge), so the two share nothing but the input vertices.
"""
import numpy as np

from . import all_element_matrices, apply_local, node_coords


class MultiBlockMesh:
    def __init__(self, mb, p):
        self.blocks, self.p = list(mb.blocks), p
        self.lo, self.hi = mb.lo, mb.hi
        n3 = (p + 1) ** 3
        self.sizes = [m.ncells * n3 for m in self.blocks]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        xyz = np.concatenate([node_coords(m, p) for m in self.blocks])
        key = np.round(xyz * 1e7).astype(np.int64)
        _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
        self.gidx = inv.reshape(-1).astype(np.int64)   # global DoF of every cell-wise entry
        self.NG = len(first)
        self.gcoords = xyz[first]                      # position of every global DoF
        self.copy_coords = xyz
        self.L = int(self.offsets[-1])

    def block_slices(self):
        return [slice(int(self.offsets[b]), int(self.offsets[b + 1])) for b in range(len(self.blocks))]

    def gather(self, ug):
        """x = G u: every copy takes its global DoF's value."""
        return np.asarray(ug, np.float64)[self.gidx]

    def scatter_add(self, y):
        """G^T y: the sum of the copies of every global DoF."""
        return np.bincount(self.gidx, weights=np.asarray(y, np.float64), minlength=self.NG)

    def dss(self, y):
        """S y = G G^T y (Sec. 4.1, Eq. (dss_operator))."""
        return self.gather(self.scatter_add(y))

    def valence(self):
        """Number of copies of every cell-wise entry's DoF (diagonal of G^T G, gathered)."""
        return self.gather(np.bincount(self.gidx, minlength=self.NG).astype(np.float64))

    def apply_local(self, kind, x):
        """y = A x block by block (cell-local, unassembled)."""
        x = np.asarray(x, np.float64)
        return np.concatenate([apply_local(m, self.p, kind, x[s]) for m, s in zip(self.blocks, self.block_slices())])

    def assemble(self, kind):
        """A_CG as a scipy CSR matrix over the global DoFs."""
        import scipy.sparse as sp
        n3 = (self.p + 1) ** 3
        rows, cols, vals = [], [], []
        for m, s in zip(self.blocks, self.block_slices()):
            A = all_element_matrices(m, self.p, kind)
            g = self.gidx[s].reshape(m.ncells, n3)
            rows.append(np.repeat(g, n3, axis=1).ravel())
            cols.append(np.tile(g, (1, n3)).ravel())
            vals.append(A.ravel())
        return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.NG, self.NG)).tocsr()

    def boundary_mask(self, tol=1e-9):
        """1 on global DoFs inside the domain cube, 0 on its boundary (homogeneous Dirichlet)."""
        c = self.gcoords
        on = np.any((np.abs(c - self.lo) < tol) | (np.abs(c - self.hi) < tol), axis=1)
        return np.where(on, 0.0, 1.0)
