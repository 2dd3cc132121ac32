"""Geometric h-multigrid V-cycle (oracle; test infrastructure).

Sec. 5.1: the Poisson solver is preconditioned by one V-cycle of a geometric
multigrid method with a Chebyshev smoother (degree 5 for pre- and
post-smoothing, smoothing range 20, eigenvalue estimates from an initial CG
run), a Chebyshev coarse solver whose degree brings the Chebyshev error
estimate to 1e-3, coarsening down to one element, and matrix-free tensorial
embedding between mother and child cells for the level transfer.

Here every level is the same structured mesh with half the cells per
direction (a direction with an odd number of cells is not coarsened) and the
same degree; its operator is the rediscretised SIPG operator of ``sipg.SIPG``
(assembled, small meshes only).  The coarse levels of a tanh-graded channel
keep the graded cell vertices but map each cell affinely ("channel_linear"):
a coarse cell spanning several fine layers cannot carry the degree-k
interpolant of the steep wall grading, and the V-cycle with iso-parametric
coarse cells was found to converge far worse (Sec. 7.1 meshes; the reading is
that the hierarchy is refined from a graded coarse mesh with straight cells).  Prolongation maps a coarse
polynomial to the fine cells by evaluating the coarse Lagrange basis at the
fine nodes in the coarse reference coordinates; restriction is its transpose.
"""
import numpy as np
import scipy.sparse as sp

from .basis import lagrange_values
from .mesh import MeshSpec, cell_ijk
from .sipg import SIPG
from .solvers import chebyshev_from


def coarsen_spec(spec):
    """Half the cells in every direction with an even count > 1; None if none."""
    n = list(spec.n)
    f = [2 if (v % 2 == 0 and v > 1) else 1 for v in n]
    if all(v == 1 for v in f):
        return None, f
    mapping = "channel_linear" if spec.mapping == "channel" else spec.mapping
    c = MeshSpec(n[0] // f[0], n[1] // f[1], n[2] // f[2], lo=spec.lo, hi=spec.hi, bc_lo=spec.bc_lo,
                 bc_hi=spec.bc_hi, mapping=mapping, gamma=spec.gamma)
    return c, f


def embedding_1d(zn, child, factor):
    """E[a, b] = l_b((child + z_a) / 2) for a coarsened direction, else identity."""
    p = len(zn)
    if factor == 1:
        return np.eye(p)
    return lagrange_values(zn, (child + np.asarray(zn)) / 2.0)


def prolongation(fine, coarse, f, zn):
    """Sparse P (n_fine x n_coarse): fine cell values = (E_z x E_y x E_x) parent values."""
    p = len(zn)
    P3 = p ** 3
    rows, cols, vals = [], [], []
    ii, jj = np.meshgrid(np.arange(P3), np.arange(P3), indexing="ij")
    for cell in range(fine.ncell):
        ix, iy, iz = (int(v) for v in cell_ijk(fine, cell))
        parent = ((iz // f[2]) * coarse.ny + iy // f[1]) * coarse.nx + ix // f[0]
        B = np.kron(embedding_1d(zn, iz % f[2], f[2]),
                    np.kron(embedding_1d(zn, iy % f[1], f[1]), embedding_1d(zn, ix % f[0], f[0])))
        rows.append((cell * P3 + ii).ravel())
        cols.append((parent * P3 + jj).ravel())
        vals.append(B.ravel())
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(fine.ncell * P3, coarse.ncell * P3)).tocsr()


class Multigrid:
    """Level hierarchy with assembled SIPG Laplacians (small meshes)."""

    def __init__(self, spec, k, penalty_factor=1.0):
        self.specs, self.factors = [spec], []
        while True:
            c, f = coarsen_spec(self.specs[-1])
            if c is None:
                break
            self.specs.append(c)
            self.factors.append(f)
        self.ops = [SIPG(s, k, penalty_factor) for s in self.specs]
        self.A = [op.assemble() for op in self.ops]
        self.D = [A.diagonal() for A in self.A]
        zn = self.ops[0].zn
        self.P = [prolongation(self.specs[i], self.specs[i + 1], self.factors[i], zn)
                  for i in range(len(self.specs) - 1)]

    @property
    def nlevels(self):
        return len(self.specs)

    def vcycle(self, b, lmax, degree=5, smoothing_range=20.0, coarse_degree=10, coarse_interval=None):
        """One V-cycle x = V(b) from x = 0.  lmax[l] is the upper end of the
        spectrum of D^-1 A used on level l (smoothing interval
        [lmax/range, lmax]); the coarsest level runs ``coarse_degree``
        Chebyshev steps from zero on ``coarse_interval`` (default: the same
        smoothing interval)."""
        self._args = (lmax, degree, smoothing_range, coarse_degree, coarse_interval)
        return self._vcycle(0, np.asarray(b, dtype=np.float64))

    def _smooth(self, l, b, x0, degree, lo, hi):
        A, D = self.A[l], self.D[l]
        return chebyshev_from(lambda v: A @ v, D, b, x0, degree, lo, hi)

    def _vcycle(self, l, b):
        lmax, degree, rng, coarse_degree, coarse_interval = self._args
        if l == self.nlevels - 1:
            lo, hi = coarse_interval if coarse_interval is not None else (lmax[l] / rng, lmax[l])
            return self._smooth(l, b, None, coarse_degree, lo, hi)
        x = self._smooth(l, b, None, degree, lmax[l] / rng, lmax[l])
        r = b - self.A[l] @ x
        xc = self._vcycle(l + 1, self.P[l].T @ r)
        x = x + self.P[l] @ xc
        return self._smooth(l, b, x, degree, lmax[l] / rng, lmax[l])
