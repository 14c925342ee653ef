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

    def _needed_cells(self):
        """Sampled cells and their face neighbours (the columns their rows touch)."""
        m = self.disc.mesh
        need = set(int(c) for c in self.cells)
        for c in self.cells:
            multi = [int(v) for v in m.cell_multi(int(c))]
            for a in range(m.D):
                for dlt in (-1, 1):
                    mm = list(multi)
                    mm[a] = (mm[a] + dlt) % m.nc[a]
                    need.add(int(m.cell_flat(mm)))
        return np.array(sorted(need))

    def apply(self, y_nodal, rhs=False):
        """M^-1 D x (or M^-1 (h - D x)) in nodal form, for the assembled rows' cells."""
        d = self.disc
        if self.full:
            z = d.from_gauss_nodal(y_nodal)
        else:  # only the cells the assembled rows couple to are converted
            per = d.n * d.mesh.nloc
            z = np.zeros_like(y_nodal)
            for c in self._needed_cells():
                sl = slice(c * per, (c + 1) * per)
                z[sl] = d.from_gauss_nodal(y_nodal[sl])
        Dz = d.D @ z
        v = (d.h - Dz) if rhs else Dz
        if self.full:
            return d.to_gauss_nodal(self._Minv(v))
        out = np.zeros_like(y_nodal)
        per = d.n * d.mesh.nloc
        mv = self._Minv(v)
        for c in self.cells:
            sl = slice(c * per, (c + 1) * per)
            out[sl] = d.to_gauss_nodal(mv[sl])
        return out

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
