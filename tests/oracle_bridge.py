"""Test helpers that express the oracle's results in the library's nodal (Gauss-point) basis.

The oracle works in the paper's Lagrange basis; the library stores nodal values at the tensor
Gauss points.  With the same quadrature both discretise the same operator on the same space Q^k,
so comparisons go through the per-cell evaluation matrix E (oracle coefficients -> values at the
Gauss points): L_nodal = E M^-1 D E^-1 and s_nodal = E M^-1 h.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import dg, steppers


class NodalOracle:
    def __init__(self, prob, rows_of_cells=None):
        self.prob = prob
        self.disc = dg.Discretisation(prob, rows_of_cells=rows_of_cells)
        self.cells = self.disc.row_cells
        self.full = rows_of_cells is None
        if self.full:
            self.Mlu = spla.splu(sp.csc_matrix(self.disc.M))

    def _Minv(self, v):
        if self.full:
            return self.Mlu.solve(v)
        # block-diagonal mass matrix: invert the blocks of the assembled rows only
        d = self.disc
        out = np.zeros_like(v)
        nl = d.mesh.nloc
        for ci, c in enumerate(self.cells):
            blk = d.mass_blocks[ci]
            idx = d.dof(c, 0, 0) + np.arange(d.n * nl)
            out[idx] = np.linalg.solve(blk, v[idx].reshape(d.n, nl).T).T.ravel()
        return out

    def apply(self, y_nodal, rhs=False):
        """M^-1 D x (or M^-1 (h - D x)) in nodal form, for the assembled rows' cells."""
        d = self.disc
        z = d.from_gauss_nodal(y_nodal)
        Dz = d.D @ z
        v = (d.h - Dz) if rhs else Dz
        return d.to_gauss_nodal(self._Minv(v))

    def row_mask(self):
        d = self.disc
        m = np.zeros(d.N, dtype=bool)
        for c in self.cells:
            m[d.dof(c, 0, 0): d.dof(c, 0, 0) + d.n * d.mesh.nloc] = True
        return m

    def rk4(self, y0_nodal, dt, nsteps):
        d = self.disc
        z = steppers.rk4(d.M, d.D, d.h, d.from_gauss_nodal(y0_nodal), dt, nsteps)
        return d.to_gauss_nodal(z)

    def cn(self, y0_nodal, dt, nsteps):
        d = self.disc
        z = steppers.theta_method(d.M, d.D, d.h, d.from_gauss_nodal(y0_nodal), dt, nsteps, theta=0.5)
        return d.to_gauss_nodal(z)
