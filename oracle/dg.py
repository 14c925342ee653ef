"""Discontinuous-Galerkin discretisation of the advection--reaction system, assembled as sparse
matrices by quadrature.

TEST INFRASTRUCTURE ONLY: part of the FP64 CPU oracle (see ``oracle/__init__.py``).  It shares no
code with the CUDA library and the product path never imports it.

Follows the paper (arXiv:2501.05110) step by step:

* advection matrices beta^alpha, reaction matrix R (Sec. 2.2, Eq. definitions-advection-reaction-eq);
* the local Lax--Friedrichs flux J = 1/2 beta (f_lo + f_hi) + 1/2 alpha (f_lo - f_hi) as the
  alternative the paper names (Sec. 3.2), selected by a problem's ``flux``;
* broken tensor-product Lagrange space Q^k, equidistant nodes for k <= 2 and Gauss--Lobatto nodes
  for k > 2 (Sec. 3.1);
* weak form after integration by parts (Eq. advection-term-by-parts, Eq.
  linear-system-degrees-of-freedom) with the upwind flux J = W (L+ W^T f1 + L- W^T f2)
  (Eq. definition-upwind-flux), eigen-pairs of n.beta computed at every face point (the oracle does
  not use the "eigenvectors once" shortcut of Sec. 3.2, which is an optimisation);
* boundary fluxes: zero inflow J = W L+ W^T f (Eq. definition-boundary-flux), continuous
  J = W (L+ + L-) W^T f (Eq. continuous-bc), periodic (Sec. 2.2);
* M, D, h of Eq. definition-mass-and-dg-matrix.

Readings of points the paper leaves open:

* quadrature: Gauss--Legendre with k+1 points per axis on cells and faces; the coefficient fields
  are sampled at the quadrature points;
* ln p momentum axis: d/dp = p^-1 d/d(ln p), so beta^{ln p} = beta^p / p, the weak form uses the
  flat measure dx d(ln p), and div beta is taken in (x, ln p);
* dU/dt is the material derivative of the prescribed (static) flow, supplied by the caller as
  the field ``DUDt``;
* units q = m = c = 1: V = p / sqrt(1+p^2), gamma m = sqrt(1+p^2), omega = B / (gamma m) (Tab. 1);
  without a momentum axis V and omega are given directly;
* a periodic face samples the fields at the upper end of the axis.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from . import sh

SPATIAL = {"x": 0, "y": 1, "z": 2}


# --------------------------------------------------------------------------------------------
# 1-D building blocks (Sec. 3.1)
# --------------------------------------------------------------------------------------------
def gauss_rule(q: int):
    """Gauss--Legendre nodes and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def basis_nodes(k: int) -> np.ndarray:
    """Nodes of the paper's Lagrange basis on [0, 1]: equidistant for k <= 2, Gauss--Lobatto
    (roots of P_k' plus the end points) for k > 2 (Sec. 3.1, Eq. lagrange-polynomial)."""
    if k == 0:
        return np.array([0.5])
    if k <= 2:
        return np.linspace(0.0, 1.0, k + 1)
    dP = np.polynomial.legendre.Legendre.basis(k).deriv()
    inner = np.sort(dP.roots().real)
    return 0.5 * (np.concatenate([[-1.0], inner, [1.0]]) + 1.0)


def lagrange_eval(nodes: np.ndarray, x: np.ndarray):
    """Values and first derivatives of the Lagrange polynomials on ``nodes`` at points ``x``.

    Returns (B, dB) of shape (len(x), len(nodes)), ell_i(x) = prod_{j != i} (x - x_j)/(x_i - x_j)."""
    x = np.atleast_1d(np.asarray(x, dtype=float))
    nb = len(nodes)
    B = np.ones((len(x), nb))
    dB = np.zeros((len(x), nb))
    for i in range(nb):
        others = [j for j in range(nb) if j != i]
        den = np.prod([nodes[i] - nodes[j] for j in others]) if others else 1.0
        for p in range(len(x)):
            terms = [x[p] - nodes[j] for j in others]
            B[p, i] = np.prod(terms) / den
            d = 0.0
            for t in range(len(terms)):
                d += np.prod(terms[:t] + terms[t + 1:])
            dB[p, i] = d / den
    return B, dB


def _tensor(mats_per_axis):
    """Kronecker-style tensor product of per-axis (P_a, I_a) tables, axis 0 fastest in both
    point and function index.  Returns (prod P_a, prod I_a)."""
    out = np.ones((1, 1))
    for M in mats_per_axis:  # earlier axes vary fastest
        out = np.einsum("pi,qj->qpji", out, M).reshape(out.shape[0] * M.shape[0], out.shape[1] * M.shape[1])
    return out


# --------------------------------------------------------------------------------------------
# mesh
# --------------------------------------------------------------------------------------------
class Mesh:
    """Tensor-product mesh of the reduced phase space; cells lexicographic, axis 0 fastest."""

    def __init__(self, prob):
        self.axes = list(prob.axes)
        self.D = len(self.axes)
        self.edges = [np.asarray(e, dtype=float) for e in prob.edges]
        self.nc = [len(e) - 1 for e in self.edges]
        self.ncell = int(np.prod(self.nc))
        self.k = prob.k
        self.q = prob.k + 1
        self.nloc = self.q ** self.D

    def cell_multi(self, c):
        """Multi-index (axis 0 fastest) of flat cell index array ``c``."""
        out, rest = [], np.asarray(c)
        for a in range(self.D):
            out.append(rest % self.nc[a])
            rest = rest // self.nc[a]
        return out

    def cell_flat(self, multi):
        c, stride = 0, 1
        for a in range(self.D):
            c = c + multi[a] * stride
            stride *= self.nc[a]
        return c


# --------------------------------------------------------------------------------------------
# coefficient matrices beta^alpha and R - div(beta) at points (Sec. 2.2)
# --------------------------------------------------------------------------------------------
def _point_state(prob, coords):
    """Split point coordinates (P, D) into spatial coordinates and momentum quantities."""
    axes = list(prob.axes)
    sp_axes = [a for a in axes if a in SPATIAL]
    xs = coords[:, [axes.index(a) for a in sp_axes]] if sp_axes else np.zeros((coords.shape[0], 0))
    mom = [a for a in axes if a in ("p", "lnp")]
    st = {"xs": xs, "mom_axis": mom[0] if mom else None}
    if mom:
        qv = coords[:, axes.index(mom[0])]
        p = np.exp(qv) if mom[0] == "lnp" else qv
        gm = np.sqrt(1.0 + p * p)
        st.update(p=p, gm=gm, V=p / gm)
        st["omega"] = prob.B(xs) / gm[:, None]
    else:
        st.update(p=None, gm=None, V=np.full(coords.shape[0], float(prob.V)))
        st["omega"] = prob.omega(xs)
    return st


def advection_matrix(prob, T, axis_kind, st, terms):
    """beta^alpha at the points of ``st``; shape (P, n, n)."""
    P, n = st["xs"].shape[0], T["n"]
    out = np.zeros((P, n, n))
    if axis_kind in SPATIAL:
        if "adv" in terms:
            a = SPATIAL[axis_kind]
            U = prob.U(st["xs"])
            out += U[:, a, None, None] * np.eye(n) + st["V"][:, None, None] * T["A"][a]
        return out
    if "mom" in terms:  # beta^p = -gamma m dU_a/dt A^a - p dU_b/dx^a A^a A^b  (Eq. beta-p)
        DU = prob.DUDt(st["xs"])
        G = prob.gradU(st["xs"])  # G[:, a, b] = dU_b / dx^a
        for a in range(3):
            out -= (st["gm"] * DU[:, a])[:, None, None] * T["A"][a]
            for b in range(3):
                out -= (st["p"] * G[:, a, b])[:, None, None] * T["AA"][a, b]
        if axis_kind == "lnp":
            out /= st["p"][:, None, None]
    return out


def reaction_minus_div(prob, T, st, terms):
    """R - div(beta) at the points of ``st``; shape (P, n, n)  (Eq. linear-system-degrees-of-freedom)."""
    P, n = st["xs"].shape[0], T["n"]
    R = np.zeros((P, n, n))
    I = np.eye(n)
    if "mom" in terms:
        DU = prob.DUDt(st["xs"])
        G = prob.gradU(st["xs"])
        for a in range(3):
            R += (DU[:, a] / st["V"])[:, None, None] * T["E"][a]
            for b in range(3):
                R += G[:, a, b][:, None, None] * T["F"][a, b]
    if "rot" in terms:
        for a in range(3):
            R -= st["omega"][:, a][:, None, None] * T["Om"][a]
    if "coll" in terms:
        R += prob.nu(st["xs"], st["p"])[:, None, None] * T["C"]
    # divergence of the advection matrices over the resolved axes
    div = np.zeros((P, n, n))
    if "adv" in terms:
        G = prob.gradU(st["xs"])
        for ax in prob.axes:
            if ax in SPATIAL:
                a = SPATIAL[ax]
                div += G[:, a, a][:, None, None] * I
    if "mom" in terms and st["mom_axis"] is not None:
        DU = prob.DUDt(st["xs"])
        G = prob.gradU(st["xs"])
        if st["mom_axis"] == "p":  # d/dp beta^p, with d(gamma m)/dp = V
            for a in range(3):
                div -= (st["V"] * DU[:, a])[:, None, None] * T["A"][a]
                for b in range(3):
                    div -= G[:, a, b][:, None, None] * T["AA"][a, b]
        else:  # p d/dp (beta^p / p) = DU_a/dt A^a / (gamma m p)
            for a in range(3):
                div += (DU[:, a] / (st["gm"] * st["p"]))[:, None, None] * T["A"][a]
    return R - div


def upwind_split(beta, flux="upwind"):
    """The face flux J = K_+ f_lo + K_- f_hi for stacked symmetric matrices beta (P, n, n):
    upwind (Eq. definition-upwind-flux): K_+- = W L+- W^T, the positive / negative eigen-parts;
    local Lax--Friedrichs (Sec. 3.2): K_+- = (beta +- alpha 1) / 2 with alpha the largest |eigenvalue|
    at the point, i.e. J = 1/2 beta (f_lo + f_hi) + 1/2 alpha (f_lo - f_hi)."""
    lam, W = np.linalg.eigh(beta)
    if flux == "llf":
        alpha = np.abs(lam).max(axis=1)
        eye = np.eye(beta.shape[1])[None]
        return 0.5 * (beta + alpha[:, None, None] * eye), 0.5 * (beta - alpha[:, None, None] * eye)
    lp = np.where(lam > 0, lam, 0.0)
    lm = np.where(lam < 0, lam, 0.0)
    bp = np.einsum("pij,pj,pkj->pik", W, lp, W)
    bm = np.einsum("pij,pj,pkj->pik", W, lm, W)
    # eigh mixes rounding residue (~1e-17 |beta|) into entries that vanish exactly by symmetry;
    # drop entries below 1e-14 |beta| so the sparsity pattern stays that of the exact matrices
    scale = np.abs(beta).max(axis=(1, 2), keepdims=True)
    bp[np.abs(bp) < 1e-14 * scale] = 0.0
    bm[np.abs(bm) < 1e-14 * scale] = 0.0
    return bp, bm


# --------------------------------------------------------------------------------------------
# assembly
# --------------------------------------------------------------------------------------------
class Discretisation:
    """Sparse M, D, h of Eq. definition-mass-and-dg-matrix for one problem.

    ``rows_of_cells`` restricts assembly to the rows of the given cells (for sampled checks on
    meshes too large to assemble); columns are always global."""

    def __init__(self, prob, rows_of_cells=None):
        self.prob = prob
        self.mesh = Mesh(prob)
        self.T = sh.tables(prob.lmax)
        self.n = self.T["n"]
        self.terms = set(prob.terms)
        m = self.mesh
        self.N = m.ncell * self.n * m.nloc
        self.row_cells = np.arange(m.ncell) if rows_of_cells is None else np.asarray(rows_of_cells)
        self.row_mask = np.zeros(m.ncell, dtype=bool)
        self.row_mask[self.row_cells] = True
        # 1-D tables on the reference interval [0,1]
        self.xg, self.wg = gauss_rule(m.q)
        self.nodes = basis_nodes(m.k)
        self.Bq, self.dBq = lagrange_eval(self.nodes, self.xg)
        self.B0, _ = lagrange_eval(self.nodes, np.array([0.0]))
        self.B1, _ = lagrange_eval(self.nodes, np.array([1.0]))
        self._assemble()

    # DoF numbering: ((cell * n + r) * nloc + a)
    def dof(self, cell, r, a):
        return (cell * self.n + r) * self.mesh.nloc + a

    def _cell_geometry(self, cells):
        m = self.mesh
        multi = m.cell_multi(cells)
        lo = np.stack([m.edges[a][multi[a]] for a in range(m.D)], axis=1)
        h = np.stack([m.edges[a][multi[a] + 1] - m.edges[a][multi[a]] for a in range(m.D)], axis=1)
        return multi, lo, h

    def _add(self, rows, cols, vals):
        keep = vals.ravel() != 0.0
        self._r.append(rows.ravel()[keep])
        self._c.append(cols.ravel()[keep])
        self._v.append(vals.ravel()[keep])

    def _assemble(self):
        m, n, T = self.mesh, self.n, self.T
        D, q, nloc = m.D, m.q, m.nloc
        self._r, self._c, self._v = [], [], []
        cells = self.row_cells
        _, lo, h = self._cell_geometry(cells)
        nC = len(cells)
        # ---- volume terms ------------------------------------------------------------------
        # quadrature point offsets and weights, axis 0 fastest
        qidx = np.array(list(itertools.product(range(q), repeat=D)))[:, ::-1]  # (nq, D), axis0 fastest
        nq = len(qidx)
        ref = self.xg[qidx]  # (nq, D)
        wref = np.prod(self.wg[qidx], axis=1)  # (nq,)
        coords = lo[:, None, :] + h[:, None, :] * ref[None]  # (nC, nq, D)
        W = wref[None, :] * np.prod(h, axis=1)[:, None]  # (nC, nq)
        Phi = _tensor([self.Bq] * D)  # (nq, nloc)
        dPhi_ref = []
        for a in range(D):
            dPhi_ref.append(_tensor([self.dBq if b == a else self.Bq for b in range(D)]))
        st = _point_state(self.prob, coords.reshape(-1, D))
        Rv = reaction_minus_div(self.prob, T, st, self.terms).reshape(nC, nq, n, n)
        betas = [advection_matrix(self.prob, T, ax, st, self.terms).reshape(nC, nq, n, n) for ax in m.axes]
        pairs = np.argwhere((np.abs(Rv).max(axis=(0, 1)) > 0) | np.any([np.abs(b).max(axis=(0, 1)) > 0 for b in betas], axis=0))
        a_idx = np.arange(nloc)
        for (r, s) in pairs:
            blk = np.einsum("cq,qa,qb->cab", W * Rv[:, :, r, s], Phi, Phi)
            for a in range(D):
                blk -= np.einsum("cq,qa,qb->cab", W * betas[a][:, :, r, s] / h[:, a:a + 1], dPhi_ref[a], Phi)
            rows = self.dof(cells[:, None, None], r, a_idx[None, :, None])
            cols = self.dof(cells[:, None, None], s, a_idx[None, None, :])
            self._add(np.broadcast_to(rows, blk.shape), np.broadcast_to(cols, blk.shape), blk)
        # mass matrix and load vector
        mass = np.einsum("cq,qa,qb->cab", W, Phi, Phi)
        self.mass_blocks = mass  # per assembled cell (same block for every coefficient)
        self._mr, self._mc, self._mv = [], [], []
        for r in range(n):
            rows = self.dof(cells[:, None, None], r, a_idx[None, :, None])
            cols = self.dof(cells[:, None, None], r, a_idx[None, None, :])
            self._mr.append(np.broadcast_to(rows, mass.shape).ravel())
            self._mc.append(np.broadcast_to(cols, mass.shape).ravel())
            self._mv.append(mass.ravel())
        self.h = np.zeros(self.N)
        if "src" in self.terms:
            s000 = self.prob.s000(st["xs"], st["p"]).reshape(nC, nq)
            load = np.einsum("cq,qa->ca", W * s000, Phi)
            self.h[self.dof(cells[:, None], 0, a_idx[None, :])] = load
        # ---- face terms --------------------------------------------------------------------
        for ax in range(D):
            self._assemble_faces(ax)
        Nn = self.N

        def cat(parts, dtype):  # no entries at all is valid: e.g. l_max = 0 with U = 0 gives D = 0
            return np.concatenate(parts) if parts else np.zeros(0, dtype=dtype)

        self.D = sp.csr_matrix((cat(self._v, float), (cat(self._r, np.int64), cat(self._c, np.int64))), shape=(Nn, Nn))
        self.M = sp.csr_matrix((cat(self._mv, float), (cat(self._mr, np.int64), cat(self._mc, np.int64))), shape=(Nn, Nn))
        del self._r, self._c, self._v, self._mr, self._mc, self._mv

    def _assemble_faces(self, ax):
        """Interior, periodic and boundary faces normal to axis ``ax`` (Eq. numerical-at-interface,
        Eq. sum-interface-boundaries)."""
        m, n, T = self.mesh, self.n, self.T
        D, q = m.D, m.q
        prob = self.prob
        bc_lo, bc_hi = prob.bc[ax]
        periodic = bc_lo == "periodic"
        nca = m.nc[ax]
        tang = [b for b in range(D) if b != ax]
        # tangential cell multi-indices
        tgrid = list(itertools.product(*[range(m.nc[b]) for b in tang[::-1]]))
        tgrid = np.array([t[::-1] for t in tgrid]) if tang else np.zeros((1, 0), dtype=int)
        # face quadrature (tangential Gauss points), tangential axis order as in ``tang``
        fidx = np.array(list(itertools.product(range(q), repeat=len(tang))))[:, ::-1] if tang else np.zeros((1, 0), dtype=int)
        nfq = len(fidx)
        # traces of the local basis on the upper face (xi_ax = 1) and the lower face (xi_ax = 0)
        per_axis_up = [self.B1 if b == ax else self.Bq for b in range(D)]
        per_axis_dn = [self.B0 if b == ax else self.Bq for b in range(D)]
        Tr_up = _tensor(per_axis_up)  # (nfq, nloc)
        Tr_dn = _tensor(per_axis_dn)
        a_idx = np.arange(m.nloc)
        for f in range(nca + 1):
            if periodic and f == 0:
                continue
            lo_i = f - 1 if f >= 1 else None
            hi_i = f if f <= nca - 1 else (0 if periodic else None)
            # cells on both sides for every tangential position
            def flat(i):
                if i is None:
                    return None
                multi = [None] * D
                multi[ax] = np.full(len(tgrid), i)
                for t, b in enumerate(tang):
                    multi[b] = tgrid[:, t]
                return m.cell_flat(multi)
            c_lo, c_hi = flat(lo_i), flat(hi_i)
            keep_lo = self.row_mask[c_lo] if c_lo is not None else None
            keep_hi = self.row_mask[c_hi] if c_hi is not None else None
            if (c_lo is None or not keep_lo.any()) and (c_hi is None or not keep_hi.any()):
                continue
            # only the faces of this plane that border an assembled row (all of them without a
            # row restriction); every face point is evaluated on its own
            touch = np.zeros(len(tgrid), dtype=bool)
            if c_lo is not None:
                touch |= keep_lo
            if c_hi is not None:
                touch |= keep_hi
            tsel = np.nonzero(touch)[0]
            nt = len(tsel)
            if c_lo is not None:
                c_lo, keep_lo = c_lo[tsel], keep_lo[tsel]
            if c_hi is not None:
                c_hi, keep_hi = c_hi[tsel], keep_hi[tsel]
            # face points and weights
            ref_cell = c_lo if c_lo is not None else c_hi
            _, lo, h = self._cell_geometry(ref_cell)
            xf = m.edges[ax][f]
            coords = np.empty((nt, nfq, D))
            coords[:, :, ax] = xf
            for t, b in enumerate(tang):
                coords[:, :, b] = lo[:, b][:, None] + h[:, b][:, None] * self.xg[fidx[:, t]][None, :]
            Wf = np.prod(self.wg[fidx], axis=1)[None, :] * np.prod(h[:, tang], axis=1)[:, None] if tang else np.ones((nt, 1))
            st = _point_state(prob, coords.reshape(-1, D))
            beta = advection_matrix(prob, T, m.axes[ax], st, self.terms)
            bp, bm = upwind_split(beta, getattr(prob, "flux", "upwind"))
            beta = beta.reshape(nt, nfq, n, n)
            bp = bp.reshape(beta.shape)
            bm = bm.reshape(beta.shape)
            # J = K_lo f_lo + K_hi f_hi; lo rows get +J, hi rows get -J
            if c_lo is not None and c_hi is not None:
                K_lo, K_hi = bp, bm
            elif c_lo is not None:  # upper boundary
                K_lo = bp if bc_hi == "inflow0" else beta
                K_hi = None
            else:  # lower boundary
                K_lo = None
                K_hi = bm if bc_lo == "inflow0" else beta
            blocks = []
            if c_lo is not None and K_lo is not None:
                blocks.append((c_lo, keep_lo, +1.0, Tr_up, c_lo, Tr_up, K_lo))
                if c_hi is not None:
                    blocks.append((c_hi, keep_hi, -1.0, Tr_dn, c_lo, Tr_up, K_lo))
            if c_hi is not None and K_hi is not None:
                blocks.append((c_hi, keep_hi, -1.0, Tr_dn, c_hi, Tr_dn, K_hi))
                if c_lo is not None:
                    blocks.append((c_lo, keep_lo, +1.0, Tr_up, c_hi, Tr_dn, K_hi))
            for (crow, keep, sign, Trow, ccol, Tcol, K) in blocks:
                sel = np.nonzero(keep)[0]
                if len(sel) == 0:
                    continue
                pairs = np.argwhere(np.abs(K[sel]).max(axis=(0, 1)) > 0)
                for (r, s) in pairs:
                    blk = sign * np.einsum("cf,fa,fb->cab", Wf[sel] * K[sel][:, :, r, s], Trow, Tcol)
                    rows = self.dof(crow[sel][:, None, None], r, a_idx[None, :, None])
                    cols = self.dof(ccol[sel][:, None, None], s, a_idx[None, None, :])
                    self._add(np.broadcast_to(rows, blk.shape), np.broadcast_to(cols, blk.shape), blk)

    # ----------------------------------------------------------------------------------------
    # conversion between the oracle basis and nodal values at the Gauss points
    # ----------------------------------------------------------------------------------------
    def to_gauss_nodal(self, zeta):
        """Values of f_h at the tensor Gauss points of every cell, same layout as ``zeta``."""
        E = _tensor([self.Bq] * self.mesh.D)  # (nq, nloc)
        z = zeta.reshape(-1, self.mesh.nloc)
        return (z @ E.T).ravel()

    def from_gauss_nodal(self, y):
        E = _tensor([self.Bq] * self.mesh.D)
        z = y.reshape(-1, self.mesh.nloc)
        return np.linalg.solve(E, z.T).T.ravel()

    def gauss_points(self):
        """Physical coordinates (ncell, nq, D) of the tensor Gauss points of every cell."""
        m = self.mesh
        cells = np.arange(m.ncell)
        _, lo, h = self._cell_geometry(cells)
        qidx = np.array(list(itertools.product(range(m.q), repeat=m.D)))[:, ::-1]
        return lo[:, None, :] + h[:, None, :] * self.xg[qidx][None]


def project_initial(disc: Discretisation, f0):
    """zeta^0 from M zeta^0 = int phi . f^0 (Eq. zeta-initial-condition).

    ``f0(coords)`` returns the n coefficients of f^0 at points (P, D) -> (P, n)."""
    import scipy.sparse.linalg as spla
    m, n = disc.mesh, disc.n
    pts = disc.gauss_points()  # (ncell, nq, D)
    _, lo, h = disc._cell_geometry(np.arange(m.ncell))
    qidx = np.array(list(itertools.product(range(m.q), repeat=m.D)))[:, ::-1]
    W = np.prod(disc.wg[qidx], axis=1)[None, :] * np.prod(h, axis=1)[:, None]
    Phi = _tensor([disc.Bq] * m.D)
    fv = f0(pts.reshape(-1, m.D)).reshape(m.ncell, -1, n)  # (ncell, nq, n)
    b = np.einsum("cq,cqr,qa->cra", W, fv, Phi).ravel()
    return spla.spsolve(disc.M.tocsc(), b)


def parameter_derivative(make_problem, theta, step):
    """dD/dtheta of the assembled dG matrix D (Eq. definition-mass-and-dg-matrix) for a family of
    problems ``theta -> make_problem(theta)``, by the fourth-order Richardson central difference

        dD ~ (8 [D(theta + s) - D(theta - s)] - [D(theta + 2 s) - D(theta - 2 s)]) / (12 s).

    Used for parameters that enter D non-linearly (the shock speed U1 enters U, grad U, dU/dt and,
    through the eigen-decompositions of n.beta, the upwind splits of Eq. definition-upwind-flux).
    The upwind split |beta| has a kink where an eigenvalue changes sign; away from such points the
    difference is accurate to O(s^4).  M does not depend on the fields."""
    Ds = {k: Discretisation(make_problem(theta + k * step)).D for k in (-2, -1, 1, 2)}
    return (8.0 * (Ds[1] - Ds[-1]) - (Ds[2] - Ds[-2])) / (12.0 * step)

