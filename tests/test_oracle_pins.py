"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: values the paper prints, closed
forms, invariants, analytic solutions or limits.  A plausible mistake anywhere in the oracle (a
dropped term, a sign, a transposed operand, a wrong normalisation) fails one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla
from scipy.linalg import expm

from oracle import dg, sh, steppers
from paper_2501_05110_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _j(code):
    """'110' -> index of (l,m,s) = (1,1,0)."""
    return sh.index_map(int(code[0]), int(code[1]), int(code[2]))


# ----------------------------------------------------------------------------------------------
# real spherical harmonics (App. A)
# ----------------------------------------------------------------------------------------------
def test_real_sh_match_printed_table():
    """App. A table of Y_lms for l <= 2 (sign and normalisation conventions)."""
    rng = np.random.default_rng(0)
    t = rng.uniform(0.05, math.pi - 0.05, 50)
    f = rng.uniform(0, 2 * math.pi, 50)
    env = {"sqrt": np.sqrt, "cos": np.cos, "sin": np.sin, "pi": math.pi, "t": t, "f": f}
    n = 0
    for line in open(os.path.join(GOLD, "real_sh_table.txt")):
        if line.startswith("#") or not line.strip():
            continue
        l, m, s, expr = line.split(maxsplit=3)
        want = eval(expr, env)
        got = sh.real_Y(int(l), int(m), int(s), t, f)
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-14)
        n += 1
    assert n == 9


def test_real_sh_orthonormal_on_independent_rule():
    """int Y_i Y_j dOmega = delta_ij (App. A) on a rule unlike the oracle's (Gauss-Chebyshev in
    theta, odd phi count)."""
    L = 6
    nt, nf = 40, 31
    # Gauss-Legendre in theta with sin(theta) weight (not in mu) + uniform phi
    x, w = np.polynomial.legendre.leggauss(nt)
    th = 0.5 * math.pi * (x + 1)
    wt = 0.5 * math.pi * w * np.sin(th)
    ph = 2 * math.pi * (np.arange(nf) + 0.3) / nf
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    Wt = np.outer(wt, np.full(nf, 2 * math.pi / nf))
    Y = np.array([sh.real_Y(l, m, s, TH, PH).ravel() for (l, m, s) in sh.lms_list(L)])
    G = (Y * Wt.ravel()) @ Y.T
    np.testing.assert_allclose(G, np.eye(len(Y)), atol=2e-9)


def test_index_map_order():
    """Eq. ordering-expansion-coefficients: (f000, f110, f100, f111, f220, f210, f200, f211, f221)."""
    want = [(0, 0, 0), (1, 1, 0), (1, 0, 0), (1, 1, 1), (2, 2, 0), (2, 1, 0), (2, 0, 0), (2, 1, 1), (2, 2, 1)]
    assert sh.lms_list(2) == want


# ----------------------------------------------------------------------------------------------
# coupling matrices (Sec. 2.1)
# ----------------------------------------------------------------------------------------------
def _closed_form_Ax_Omx(lmax):
    idx = sh.lms_list(lmax)
    n = len(idx)
    A, O = np.zeros((n, n)), np.zeros((n, n))
    for i, (lp, mp, sp) in enumerate(idx):
        for j, (l, m, s) in enumerate(idx):
            if mp == m and sp == s:
                if lp == l + 1:
                    A[i, j] = math.sqrt((l + m + 1) * (l - m + 1) / ((2 * l + 3) * (2 * l + 1)))
                if lp == l - 1:
                    A[i, j] = math.sqrt((l + m) * (l - m) / ((2 * l + 1) * (2 * l - 1)))
            if lp == l and mp == m:
                O[i, j] = m * ((sp == 0 and s == 1) / math.sqrt(1 + (mp == 0))
                               - (sp == 1 and s == 0) / math.sqrt(1 + (m == 0)))
    return A, O


@pytest.mark.parametrize("lmax", [1, 3, 5, 7])
def test_Ax_Omx_closed_forms(lmax):
    """Eq. representation-matrix-Ax and Eq. representation-matrix-Omegax."""
    T = sh.tables(lmax)
    A, O = _closed_form_Ax_Omx(lmax)
    np.testing.assert_allclose(T["A"][0], A, atol=1e-13)
    np.testing.assert_allclose(T["Om"][0], O, atol=1e-13)


def _u(lp, mp, l, m):
    """Eq. complex-rotation; the sum runs over all k with non-negative factorial arguments."""
    if lp != l:
        return 0.0
    tot = 0.0
    for k in range(2 * l + 2):
        args = (k, l - mp - k, l - m - k, mp + m + k)
        if min(args) < 0:
            continue
        tot += (-1) ** k * math.sqrt(math.factorial(l + mp) * math.factorial(l - mp) * math.factorial(l + m)
                                     * math.factorial(l - m)) / math.prod(math.factorial(a) for a in args)
    return (-1) ** (l - mp) / 2 ** l * tot


@pytest.mark.parametrize("lmax", [1, 3, 5])
def test_rotation_relations(lmax):
    """Eq. real-direction-op-matrices-and-rotations and the printed rotation elements
    (Eq. representation-matrix-Uz with Eq. complex-rotation).  The printed element formula of
    Eq. representation-matrix-Ux equals exp(-pi/2 Omega^x) (the reading taken for that element)."""
    T = sh.tables(lmax)
    A, Om = T["A"], T["Om"]
    Uz, Ux = expm(0.5 * math.pi * Om[2]), expm(0.5 * math.pi * Om[0])
    np.testing.assert_allclose(Uz.T @ A[0] @ Uz, A[1], atol=1e-12)
    np.testing.assert_allclose(Ux.T @ A[1] @ Ux, A[2], atol=1e-12)
    np.testing.assert_allclose(Uz.T @ Om[0] @ Uz, Om[1], atol=1e-12)
    np.testing.assert_allclose(Ux.T @ Om[1] @ Ux, Om[2], atol=1e-12)
    idx = sh.lms_list(lmax)
    n = len(idx)
    Uz_p, Ux_p = np.zeros((n, n)), np.zeros((n, n))
    for i, (lp, mp, sp) in enumerate(idx):
        for j, (l, m, s) in enumerate(idx):
            if sp == 0 and s == 0:
                Uz_p[i, j] = (_u(lp, mp, l, m) + (-1) ** m * _u(lp, mp, l, -m)) / math.sqrt((1 + (mp == 0)) * (1 + (m == 0)))
            if sp == 1 and s == 1:
                Uz_p[i, j] = _u(lp, mp, l, m) - (-1) ** m * _u(lp, mp, l, -m)
            if lp == l and mp == m:
                c, si = math.cos(0.5 * math.pi * m), math.sin(0.5 * math.pi * m)
                v = 0.0
                if sp == 0 and s == 0:
                    v += (c + (mp == 0 and m == 0)) / math.sqrt((1 + (mp == 0)) * (1 + (m == 0)))
                if sp == 1 and s == 0:
                    v += si / math.sqrt(1 + (mp == 0))
                if sp == 0 and s == 1:
                    v -= si / math.sqrt(1 + (m == 0))
                if sp == 1 and s == 1:
                    v += c
                Ux_p[i, j] = v
    np.testing.assert_allclose(Uz_p, Uz, atol=1e-12)
    np.testing.assert_allclose(Ux_p, Ux.T, atol=1e-12)


@pytest.mark.parametrize("lmax", [1, 2, 3, 5])
def test_matrix_invariants(lmax):
    """A symmetric, Omega antisymmetric (Sec. 2.1); sum_a A^a A^a = 1 (|p_hat| = 1, products at
    L = lmax+1); [Om^x, Om^y] = -Om^z cyclic (rotation generators); A^y, A^z share A^x's spectrum
    (Sec. 3.2); C = diag(l(l+1)/2) (Eq. real-C-matrix); A^a A^b symmetric and = A^b A^a."""
    T = sh.tables(lmax)
    A, Om, AA, n = T["A"], T["Om"], T["AA"], T["n"]
    for a in range(3):
        np.testing.assert_allclose(A[a], A[a].T, atol=1e-14)
        np.testing.assert_allclose(Om[a], -Om[a].T, atol=1e-14)
        for b in range(3):
            np.testing.assert_allclose(AA[a, b], AA[a, b].T, atol=1e-13)
            np.testing.assert_allclose(AA[a, b], AA[b, a], atol=1e-13)
    np.testing.assert_allclose(AA[0, 0] + AA[1, 1] + AA[2, 2], np.eye(n), atol=1e-13)
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        np.testing.assert_allclose(Om[a] @ Om[b] - Om[b] @ Om[a], -Om[c], atol=1e-12)
    ev = np.sort(np.linalg.eigvalsh(A[0]))
    for a in (1, 2):
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(A[a])), ev, atol=1e-12)
    np.testing.assert_allclose(np.diag(T["C"]), [l * (l + 1) / 2 for (l, m, s) in sh.lms_list(lmax)])


@pytest.mark.parametrize("lmax", [1, 3, 5])
def test_Ax_block_spectrum_is_legendre_roots(lmax):
    """The (m,s) block of A^x is the Jacobi matrix of the associated Legendre functions, so its
    eigenvalues are the roots of d^m P_{lmax+1} / dx^m (lmax = 1, m = 0: +-1/sqrt(3), Sec. 4.1)."""
    T = sh.tables(lmax)
    idx = sh.lms_list(lmax)
    for m in range(lmax + 1):
        rows = [sh.index_map(l, m, 0) for l in range(m, lmax + 1)]
        blk = T["A"][0][np.ix_(rows, rows)]
        P = np.polynomial.legendre.Legendre.basis(lmax + 1).deriv(m)
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(blk)), np.sort(P.roots().real), atol=1e-12)
    if lmax == 1:
        assert abs(np.max(np.linalg.eigvalsh(T["A"][0])) - 1 / math.sqrt(3)) < 1e-14


def test_worked_shock_system_lmax1():
    """Entries of the printed l_max = 1 shock system (Sec. 4.4, Eq. actual-soe-for-sapphire)."""
    T = sh.tables(1)
    mats = {"Ax": T["A"][0], "AxAx": T["AA"][0, 0], "Ex": T["E"][0], "Fxx": T["F"][0, 0]}
    for line in open(os.path.join(GOLD, "shock_lmax1_system.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, r, c, v = line.split()
        assert abs(mats[name][_j(r), _j(c)] - float(v)) < 1e-13, (name, r, c)
    # f_110, f_111 decouple from (f_000, f_100) for fields along x (Sec. 4.4)
    for M in mats.values():
        for a in ("000", "100"):
            for b in ("110", "111"):
                assert M[_j(a), _j(b)] == 0.0 and M[_j(b), _j(a)] == 0.0
    # the full R - div(beta) and beta^p at one point reduce to the printed 2x2 blocks
    prob = W.shock(nx=4, npc=2, lmax=1)
    xs = np.array([[0.3]])
    p = np.array([2.0])
    st = {"xs": xs, "mom_axis": "p", "p": p, "gm": np.sqrt(1 + p * p), "V": p / np.sqrt(1 + p * p),
          "omega": prob.B(xs) / np.sqrt(1 + p * p)[:, None]}
    terms = {"mom", "rot", "coll"}
    R = dg.reaction_minus_div(prob, T, st, terms)[0]
    dudx = prob.gradU(xs)[0, 0, 0]
    Du = prob.DUDt(xs)[0, 0]
    nu = prob.nu(xs, p)[0]
    V, gm = st["V"][0], st["gm"][0]
    # R itself (printed) plus div(beta^p) = -V Du A^x - dudx A^xA^x (linear p axis)
    div = -V * Du * T["A"][0] - dudx * T["AA"][0, 0]
    Rp = R + div
    i0, i1 = _j("000"), _j("100")
    np.testing.assert_allclose(Rp[np.ix_([i0, i1], [i0, i1])],
                               [[0.0, -2 / (math.sqrt(3) * V) * Du], [0.0, nu - 0.4 * dudx]], atol=1e-14)
    bp = dg.advection_matrix(prob, T, "p", st, terms)[0]
    np.testing.assert_allclose(bp[np.ix_([i0, i1], [i0, i1])],
                               -np.array([[p[0] / 3 * dudx, gm / math.sqrt(3) * Du],
                                          [gm / math.sqrt(3) * Du, 3 * p[0] / 5 * dudx]]), atol=1e-14)


# ----------------------------------------------------------------------------------------------
# whole discretisation: convergence study with its closed-form solution (Sec. 4.1)
# ----------------------------------------------------------------------------------------------
def _convergence_problem(nc, k, Lbox=20.0):
    omega, V = math.pi, math.sqrt(3) / 2  # B = 2 pi e_z, gamma = 2
    kk = 2 * math.pi / Lbox
    c1 = V * kk / math.sqrt(3)
    s1 = math.sqrt(omega ** 2 + c1 ** 2)

    def f0(c):  # A_0 = 2, B_1 = 1 (Eq. convergence-study-initial-condition-f000)
        out = np.zeros((c.shape[0], 4))
        out[:, 0] = 2 * omega - s1 * np.sin(kk * c[:, 0])
        return out

    def exact000(t, x):  # Eq. convergence-study-analytical-solution-isotropic-part
        return 2 * omega + (c1 ** 2 / s1) * (np.cos(s1 * t) - 1 + s1 ** 2 / c1 ** 2) * (-np.sin(kk * x))

    prob = W.Problem(name="conv", axes=("x",), edges=[np.linspace(0, Lbox, nc + 1)], k=k, lmax=1,
                     bc=[("periodic", "periodic")], terms=frozenset({"adv", "rot"}),
                     U=W._const3([0, 0, 0]), gradU=W._zero33, DUDt=W._const3([0, 0, 0]),
                     omega=W._const3([0, 0, omega]), V=V, nu=W._scalar(0.0), s000=W._scalar(0.0), f0=f0)
    return prob, exact000


def _rel_l2_000(disc, z, exact, t, k, nc, Lbox=20.0):
    y = disc.to_gauss_nodal(z).reshape(nc, 4, k + 1)[:, 0, :]
    x = disc.gauss_points()[:, :, 0]
    w = dg.gauss_rule(k + 1)[1] * (Lbox / nc)
    return math.sqrt(np.sum(w * (y - exact(t, x)) ** 2)) / math.sqrt(np.sum(w * y ** 2))


# meshes and RK4 steps of the space-order study per degree: the time error stays below the space
# error (dt = 0.001 for k = 5, whose finest error is ~3e-12)
CONV_SPACE = {1: ((8, 16, 32), 0.005), 2: ((8, 16, 32), 0.005), 3: ((8, 16, 32), 0.005),
              4: ((4, 8, 16, 32), 0.005), 5: ((4, 8, 16, 32), 0.001)}
CONV_FINEST = {1: 5e-4, 2: 2e-5, 3: 1e-6, 4: 2e-9, 5: 1e-11}


def convergence_order(ncs, errs):
    """Least-squares slope of log(err) against log(1/nc)."""
    return -np.polyfit(np.log(np.asarray(ncs, float)), np.log(np.asarray(errs)), 1)[0]


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_convergence_study_space(k):
    """ERK4, Delta t small: the error against the closed form falls as Delta x^(k+1) (Sec. 4.1; the
    paper runs k = 1..5).  For k >= 4 the mesh-to-mesh orders oscillate about k+1 (6.1, 5.4, 6.9 for
    k = 5), so the least-squares slope over the meshes is checked."""
    ncs, dt = CONV_SPACE[k]
    errs = []
    for nc in ncs:
        prob, ex = _convergence_problem(nc, k)
        disc = dg.Discretisation(prob)
        z = steppers.rk4(disc.M, disc.D, disc.h, dg.project_initial(disc, prob.f0), dt, int(round(1.0 / dt)))
        errs.append(_rel_l2_000(disc, z, ex, 1.0, k, nc))
    assert convergence_order(ncs, errs) > k + 1 - 0.3, errs
    assert errs[-1] < CONV_FINEST[k], errs


@pytest.mark.parametrize("theta,order", [(0.5, 2), (1.0, 1), (0.0, 1)])
def test_convergence_study_time(theta, order):
    """theta-method time error orders: CN 2, backward/forward Euler 1 (Sec. 4.1, Eq. theta-method),
    error measured as the maximum over all steps of the relative L2 error of f_000."""
    k, nc, tF = 4, 16, 2.0
    prob, ex = _convergence_problem(nc, k)
    disc = dg.Discretisation(prob)
    z0 = dg.project_initial(disc, prob.f0)
    errs = []
    dts = (0.004, 0.002, 0.001) if theta == 0.0 else (0.04, 0.02, 0.01)
    for dt in dts:
        worst = [0.0]

        def cb(i, z, dt=dt):
            worst[0] = max(worst[0], _rel_l2_000(disc, z, ex, i * dt, k, nc))
        steppers.theta_method(disc.M, disc.D, disc.h, z0, dt, int(round(tF / dt)), theta=theta, callback=cb)
        errs.append(worst[0])
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(o - order) < 0.25 for o in orders), (errs, orders)


# ----------------------------------------------------------------------------------------------
# invariants and limits of the 1-D periodic advection--collision run
# ----------------------------------------------------------------------------------------------
def test_particle_number_conservation_periodic():
    """Periodic, grad U = 0: int f_000 dx is conserved (fluxes telescope, C_00 = 0, row 0 of
    Omega vanishes): the f_000 rows of D sum to zero over every column."""
    for prob in (W.periodic_1d(ncells=16), W.box3d(ncells=2, lmax=2, k=1)):
        disc = dg.Discretisation(prob)
        e = np.zeros(disc.N)
        for c in range(disc.mesh.ncell):
            e[disc.dof(c, 0, np.arange(disc.mesh.nloc))] = 1.0
        assert np.abs(disc.D.T @ e).max() < 1e-13


def test_diffusion_limit():
    """Long-wavelength f_000 mode decays at kappa k^2 with kappa = V^2 / (3 nu) (Sec. 4.4 text,
    diffusion approximation); the relative error falls ~4x when the wavelength doubles."""
    nu, V = 2.0, 1.0
    kappa = V * V / (3 * nu)
    rel = []
    for Lbox in (20.0, 40.0):
        kk = 2 * math.pi / Lbox
        prob = W.periodic_1d(ncells=32, k=2, lmax=5, U=0.0, nu=nu, V=V, L=Lbox)
        disc = dg.Discretisation(prob)
        prob.f0 = W._iso_f0(lambda c: 1.0 + 0.1 * np.cos(kk * c[:, 0]), prob.n)
        z = dg.project_initial(disc, prob.f0)
        x = disc.gauss_points()[:, :, 0].ravel()
        amps = []
        t_skip, t_meas = 10.0, 40.0  # let the fast (l >= 1) modes die out first
        for (t0, t1) in ((0.0, t_skip), (t_skip, t_skip + t_meas)):
            z = steppers.theta_method(disc.M, disc.D, disc.h, z, 0.05, int(round((t1 - t0) / 0.05)))
            y = disc.to_gauss_nodal(z).reshape(-1, prob.n, 3)[:, 0, :].ravel()
            amps.append(np.sum(y * np.cos(kk * x)))
        rate = -math.log(amps[1] / amps[0]) / t_meas
        rel.append(abs(rate / (kappa * kk * kk) - 1))
    assert rel[0] < 0.05 and rel[1] < rel[0] / 3, rel


def test_free_streaming_fourier_solution():
    """nu = 0, omega = 0: the dG solution converges to the exact solution of the truncated PDE,
    exp(-i k V A^x t) on each Fourier mode (free streaming along x)."""
    errs = []
    for nc in (16, 32):
        Lbox, V = 20.0, 1.0
        kk = 2 * math.pi / Lbox
        prob = W.periodic_1d(ncells=nc, k=2, lmax=3, U=0.0, nu=0.0, V=V, L=Lbox)
        prob.f0 = W._iso_f0(lambda c: np.cos(kk * c[:, 0]), prob.n)
        disc = dg.Discretisation(prob)
        t = 3.0
        z = steppers.rk4(disc.M, disc.D, disc.h, dg.project_initial(disc, prob.f0), 0.01, 300)
        y = disc.to_gauss_nodal(z).reshape(nc, prob.n, 3)
        x = disc.gauss_points()[:, :, 0]
        T = sh.tables(3)
        # f(x,t) = Re[ exp(-i k V A^x t) e_0 exp(i k x) ]
        G = expm(-1j * kk * V * T["A"][0] * t)[:, 0]
        want = np.real(G[None, :, None] * np.exp(1j * kk * x)[:, None, :])
        errs.append(np.abs(y - want).max())
    assert errs[1] < errs[0] / 6 and errs[1] < 2e-4, errs


# ----------------------------------------------------------------------------------------------
# parallel shock: power-law slope and normalisation (Sec. 4.4)
# ----------------------------------------------------------------------------------------------
def _graded_edges(xl, xr, Ls, dxs, grow):
    inner = np.arange(-Ls, Ls + 1e-12, dxs)
    right, d = [inner[-1]], dxs
    while right[-1] < xr:
        d *= grow
        right.append(right[-1] + d)
    left, d = [inner[0]], dxs
    while left[-1] > xl:
        d *= grow
        left.append(left[-1] - d)
    return np.concatenate([left[::-1][:-1], inner, right[1:]])


def test_shock_steady_state_slope_and_normalisation():
    """Steady state D zeta = h at a thin shock: downstream f ~ p^(-3r/(r-1)) (Eq.
    particle-spectrum-shock-rest-frame) with normalisation 3 Q / (U1 - U2); the deviation of the
    slope from -4 is first order in U1/V (it halves when U1 halves)."""
    r, Ls, sig_lnp, npc, lnp_hi = 4.0, 0.05, 0.15, 40, 6.0
    dev = []
    for U1 in (0.1, 0.05):
        xe = _graded_edges(-40 * 0.1 / U1, 120 * 0.1 / U1, Ls, 0.0125, 1.15)
        prob = W.shock(x_edges=xe, npc=npc, lnpr=(0.0, lnp_hi), lmax=1, U1=U1, r=r, Ls=Ls,
                       nu_field=lambda xs, p: np.ones(xs.shape[0]), sig_x=0.05, sig_lnp=sig_lnp, lnp0=1.0)
        disc = dg.Discretisation(prob)
        z = spla.spsolve(disc.D.tocsc(), disc.h)
        nx = len(xe) - 1
        y = disc.to_gauss_nodal(z).reshape(npc, nx, disc.n, 4)
        fbar = y[:, :, 0, :].mean(axis=2)
        xc = 0.5 * (xe[1:] + xe[:-1])
        lpc = np.linspace(0, lnp_hi, npc + 1)
        lpc = 0.5 * (lpc[1:] + lpc[:-1])
        fd = fbar[:, (xc > 2) & (xc < 20)].mean(axis=1)
        sel = (lpc > 2.0) & (lpc < 4.5)
        slope = np.polyfit(lpc[sel], np.log(fd[sel]), 1)[0]
        dev.append(abs(slope + 3 * r / (r - 1)))
        # normalisation: f_000 = sqrt(4 pi) 3 Q/(U1-U2) <(p/p0)^-4>, p0 log-normal (sigma)
        dl = lnp_hi / npc
        cellavg = (np.exp(-4 * (lpc - dl / 2)) - np.exp(-4 * (lpc + dl / 2))) / (4 * dl)
        pred = math.sqrt(4 * math.pi) * 3 * 0.1 / (U1 - U1 / r) * math.exp(8 * sig_lnp ** 2) * math.exp(4.0) * cellavg
        ratio = (fd[sel] / pred[sel])[:3]  # nearest p0; further out the O(U1/V) slope shift adds up
        assert np.all(np.abs(ratio - 1) < 0.4 * U1 + 0.01), ratio
    assert dev[0] < 0.5 * 0.1 and dev[1] < 0.5 * 0.05, dev
    assert 1.5 < dev[0] / dev[1] < 2.5, dev


# ----------------------------------------------------------------------------------------------
# solvers
# ----------------------------------------------------------------------------------------------
def test_gmres_matches_direct_solve():
    prob = W.shock(nx=16, npc=8)
    disc = dg.Discretisation(prob)
    A = disc.M + 0.5 * disc.D
    rng = np.random.default_rng(1)
    b = rng.standard_normal(disc.N)
    x_direct = spla.spsolve(A.tocsc(), b)
    x, its = steppers.gmres(A, b, np.zeros_like(b), tol=1e-12, restart=30)
    assert np.linalg.norm(A @ x - b) <= 1.01e-12 * np.linalg.norm(b)
    np.testing.assert_allclose(x, x_direct, rtol=0, atol=1e-9 * np.abs(x_direct).max())
    assert 0 < its < 200


def test_lmax0_reductions():
    """l_max = 0 keeps only f_000: A^a couples l = 0 to l = 1 only and the collision rate
    nu l(l+1)/2 vanishes at l = 0 (Sec. 2.1).  (a) 1-D periodic, constant U > 0, k = 0: the dG
    operator is first-order upwind finite volumes, M^-1 D = (U/h)(I - S) with S the periodic shift
    i-1 -> i.  (b) 3-D box with U = 0: D = 0 exactly."""
    U, nc = 0.3, 7
    prob = W.periodic_1d(ncells=nc, k=0, lmax=0, U=U)
    d = dg.Discretisation(prob)
    h = 20.0 / nc
    got = spla.spsolve(d.M.tocsc(), d.D.toarray())
    S = np.roll(np.eye(nc), 1, axis=0)  # (S z)_i = z_{i-1}
    np.testing.assert_allclose(got, (U / h) * (np.eye(nc) - S), rtol=0, atol=1e-14)
    box = dg.Discretisation(W.box3d(ncells=2, k=2, lmax=0))
    assert box.D.nnz == 0 and box.N == 8 * 27


@pytest.mark.parametrize("case", ["shock2d", "box3d"])
def test_rows_of_cells_subset_matches_full_assembly(case):
    """Assembling only the rows of some cells (faces evaluated only where they border those
    cells) reproduces those rows of the full assembly: 2-D shock with boundaries, 3-D periodic box
    (two tangential axes per face plane, wrap-around neighbours)."""
    if case == "shock2d":
        prob, cells = W.shock(nx=8, npc=6), np.array([0, 7, 9, 22, 47])
    else:
        prob, cells = W.box3d(ncells=4, k=1, lmax=2), np.array([0, 5, 21, 42, 63])
    full = dg.Discretisation(prob)
    part = dg.Discretisation(prob, rows_of_cells=cells)
    rows = np.concatenate([full.dof(c, 0, 0) + np.arange(full.n * full.mesh.nloc) for c in cells])
    np.testing.assert_allclose(part.D[rows].toarray(), full.D[rows].toarray(), atol=1e-15)
    np.testing.assert_allclose(part.M[rows].toarray(), full.M[rows].toarray(), atol=1e-15)
    np.testing.assert_allclose(part.h[rows], full.h[rows])


def _shock_nu_family():
    """Small shock with a per-cell log-normal nu, a per-cell direction v, and discretisations of
    nu0 + t v (or of v alone as a pure collision term)."""
    rng = np.random.default_rng(3)
    base = W.shock(nx=6, npc=4, lmax=2, xr=(-12.0, 12.0), lnpr=(0.0, 3.0))
    xe, pe = base.edges
    v = rng.standard_normal((len(pe) - 1, len(xe) - 1))
    nu0, _ = W.lognormal_cell_nu(xe, pe, seed=6)

    def cellfun(vals):
        def f(xs, p):
            ix = np.clip(np.searchsorted(xe, xs[:, 0], side="right") - 1, 0, len(xe) - 2)
            ip = np.clip(np.searchsorted(pe, np.log(p), side="right") - 1, 0, len(pe) - 2)
            return vals[ip, ix]
        return f

    def disc_with(nu_fun, terms=None):
        p = W.shock(nx=6, npc=4, lmax=2, xr=(-12.0, 12.0), lnpr=(0.0, 3.0), nu_field=nu_fun)
        if terms is not None:
            p.terms = frozenset(terms)
        return dg.Discretisation(p)

    return nu0, v, cellfun, disc_with


def test_rk4_tangent_matches_trajectory_differences():
    """The oracle's RK4 tangent (d zeta^N / d nu along a per-cell direction) equals a central
    difference of its own RK4 trajectories (dt = 0.02, inside RK4's stability region for the
    spectral radius 63 of M^-1 D here; the trajectory is a polynomial in nu)."""
    nu0, v, cellfun, disc_with = _shock_nu_family()
    d0 = disc_with(nu0)
    dD = disc_with(cellfun(v), terms={"coll"}).D
    dt, nsteps = 0.02, 5
    z, dz = steppers.rk4_tangent(d0.M, d0.D, d0.h, dD, np.zeros(d0.N), dt, nsteps)
    np.testing.assert_allclose(z, steppers.rk4(d0.M, d0.D, d0.h, np.zeros(d0.N), dt, nsteps), rtol=0, atol=0)
    eps = 1e-4
    zs = []
    for sgn in (1, -1):
        d = disc_with(lambda xs, p, s=sgn: nu0(xs, p) + s * eps * cellfun(v)(xs, p))
        zs.append(steppers.rk4(d.M, d.D, d.h, np.zeros(d.N), dt, nsteps))
    fd = (zs[0] - zs[1]) / (2 * eps)
    assert np.abs(fd - dz).max() < 1e-7 * np.abs(dz).max()


def test_rk4_step_transpose_dot_product():
    """<lam, Phi x> = <Phi^T lam, x> for the linear part Phi of one RK4 step (the oracle's stage
    form with h = 0) and the transpose from the stability polynomial in L^T = D^T M^-1."""
    nu0, _, _, disc_with = _shock_nu_family()
    d = disc_with(nu0)
    Mlu = spla.splu(d.M.tocsc())
    LT = lambda x: d.D.T @ Mlu.solve(x)
    rng = np.random.default_rng(8)
    for dt in (0.02, 0.5):
        x, lam = rng.standard_normal(d.N), rng.standard_normal(d.N)
        Phi_x = steppers.rk4(d.M, d.D, np.zeros(d.N), x, dt, 1)
        a, b = lam @ Phi_x, steppers.rk4_step_transpose(LT, dt, lam) @ x
        assert abs(a - b) < 1e-12 * (np.abs(lam) @ np.abs(Phi_x)), (dt, a, b)


def test_cn_tangent_matches_trajectory_differences():
    """The oracle's CN tangent (d zeta^N / d nu along a per-cell direction) equals a central
    difference of its own CN trajectories; D is linear in nu, so the difference is exact up to
    rounding."""
    rng = np.random.default_rng(3)
    base = W.shock(nx=6, npc=4, lmax=2, xr=(-12.0, 12.0), lnpr=(0.0, 3.0))
    xe, pe = base.edges
    v = rng.standard_normal((len(pe) - 1, len(xe) - 1))
    nu0, _ = W.lognormal_cell_nu(xe, pe, seed=6)

    def cellfun(vals):
        def f(xs, p):
            ix = np.clip(np.searchsorted(xe, xs[:, 0], side="right") - 1, 0, len(xe) - 2)
            ip = np.clip(np.searchsorted(pe, np.log(p), side="right") - 1, 0, len(pe) - 2)
            return vals[ip, ix]
        return f

    def disc_with(nu_fun, terms=None):
        p = W.shock(nx=6, npc=4, lmax=2, xr=(-12.0, 12.0), lnpr=(0.0, 3.0), nu_field=nu_fun)
        if terms is not None:
            p.terms = frozenset(terms)
        return dg.Discretisation(p)

    d0 = disc_with(nu0)
    dD = disc_with(cellfun(v), terms={"coll"}).D
    z, dz = steppers.cn_tangent(d0.M, d0.D, d0.h, dD, np.zeros(d0.N), 1.0, 5)
    eps = 1e-4
    zs = []
    for sgn in (1, -1):
        d = disc_with(lambda xs, p, s=sgn: nu0(xs, p) + s * eps * cellfun(v)(xs, p))
        zs.append(steppers.theta_method(d.M, d.D, d.h, np.zeros(d.N), 1.0, 5))
    fd = (zs[0] - zs[1]) / (2 * eps)
    assert np.abs(fd - dz).max() < 1e-7 * np.abs(dz).max()


def _shock_u1_family():
    def make(U1):
        return W.shock(nx=8, npc=5, lmax=2, xr=(-6.0, 6.0), lnpr=(0.0, 3.0), U1=U1, Ls=1.0)
    return make


@pytest.mark.parametrize("scheme", ["cn", "rk4"])
def test_u1_tangent_matches_trajectory_differences(scheme):
    """The oracle's tangent of the trajectory with respect to the shock speed U1 (Richardson
    difference of the assembled D fed through the CN / RK4 tangent recursions) equals a central
    difference of the oracle's own trajectories at U1 +- e.  U1 enters U, grad U, dU/dt and the
    upwind splits, so neither side is exact: the bound is the O(e^2) truncation of the trajectory
    difference.  A wrong Richardson weight (planted in a copy below) fails the same bound."""
    make = _shock_u1_family()
    u1 = 0.1
    d0 = dg.Discretisation(make(u1))
    dD = dg.parameter_derivative(make, u1, 1e-3 * u1)
    dt, nsteps = (1.0, 5) if scheme == "cn" else (0.01, 5)
    if scheme == "cn":
        _, dz = steppers.cn_tangent(d0.M, d0.D, d0.h, dD, np.zeros(d0.N), dt, nsteps)
        run = lambda d: steppers.theta_method(d.M, d.D, d.h, np.zeros(d.N), dt, nsteps)
    else:
        _, dz = steppers.rk4_tangent(d0.M, d0.D, d0.h, dD, np.zeros(d0.N), dt, nsteps)
        run = lambda d: steppers.rk4(d.M, d.D, d.h, np.zeros(d.N), dt, nsteps)
    e = 1e-4 * u1
    fd = (run(dg.Discretisation(make(u1 + e))) - run(dg.Discretisation(make(u1 - e)))) / (2 * e)
    scale = np.abs(dz).max()
    assert scale > 0
    assert np.abs(fd - dz).max() < 1e-8 * scale
    # planted mistake: a wrong Richardson weight (7 instead of 8) is detected
    Ds = {k: dg.Discretisation(make(u1 + k * 1e-3 * u1)).D for k in (-2, -1, 1, 2)}
    bad = (7.0 * (Ds[1] - Ds[-1]) - (Ds[2] - Ds[-2])) / (12.0 * 1e-3 * u1)
    if scheme == "cn":
        _, dz_bad = steppers.cn_tangent(d0.M, d0.D, d0.h, bad, np.zeros(d0.N), dt, nsteps)
    else:
        _, dz_bad = steppers.rk4_tangent(d0.M, d0.D, d0.h, bad, np.zeros(d0.N), dt, nsteps)
    assert np.abs(fd - dz_bad).max() > 1e-3 * scale


def test_c_driver_cn_matches_lu():
    """The oracle's multi-threaded C driver of the CN step (GMRES(30), right point-Jacobi, the
    algorithm of steppers.gmres) reaches the sparse-LU trajectory within its tolerance, and its
    iteration counts match the Python GMRES to within one per step (rounding order differs)."""
    from oracle import native
    prob = W.shock(nx=12, npc=6, lmax=3)
    d = dg.Discretisation(prob)
    want = steppers.theta_method(d.M, d.D, d.h, np.zeros(d.N), 1.0, 4)
    drv = native.CNDriver(d, 1.0)
    z = np.zeros(d.N)
    nt, its = drv.steps(z, 4, tol=1e-12, threads=2)
    assert nt == 2
    assert np.linalg.norm(z - want) < 1e-9 * np.linalg.norm(want)
    A = (d.M + 0.5 * d.D).tocsr()
    B = (d.M - 0.5 * d.D).tocsr()
    zp, its_py = np.zeros(d.N), 0
    for _ in range(4):
        zp, k = steppers.gmres(A, B @ zp + d.h, zp, tol=1e-12)
        its_py += k
    assert abs(its - its_py) <= 4, (its, its_py)


def test_c_driver_rk4_matches_python():
    """The C driver's RK4 step (D in CSR, inverted mass blocks, OpenMP) equals the oracle's Python RK4
    (sparse LU of M) on a 3-D box and a graded shock, to rounding."""
    from oracle import native
    for prob, dt in ((W.box3d(ncells=2, k=2, lmax=2), 0.01), (W.shock(nx=6, npc=4, lmax=3), 0.05)):
        d = dg.Discretisation(prob)
        z0 = np.random.default_rng(3).standard_normal(d.N)
        want = steppers.rk4(d.M, d.D, d.h, z0, dt, 3)
        z = z0.copy()
        assert native.RK4Driver(d).steps(z, dt, 3, threads=2) == 2
        assert np.linalg.norm(z - want) < 1e-12 * np.linalg.norm(want)


# ----------------------------------------------------------------------------------------------
# local Lax--Friedrichs flux (the alternative numerical flux of Sec. 3.2)
# ----------------------------------------------------------------------------------------------
def _with_flux(prob, flux):
    import dataclasses
    return dataclasses.replace(prob, flux=flux)


def test_llf_equals_upwind_for_scalar_advection():
    """l_max = 0: beta = U is a scalar, alpha = |U|, so the two fluxes coincide."""
    for prob in (W.periodic_1d(ncells=6, k=2, lmax=0, U=0.3), W.shock(nx=5, npc=3, lmax=0, xr=(-2.0, 2.0), lnpr=(0.0, 2.0))):
        Du = dg.Discretisation(prob).D
        Dl = dg.Discretisation(_with_flux(prob, "llf")).D
        assert abs(Du - Dl).max() < 1e-14 * abs(Du).max()


def test_llf_adds_dissipation_and_conserves():
    """alpha 1 - |beta| is positive semi-definite at every face point, so x^T (D_llf - D_up) x >= 0
    (LLF is at least as dissipative); both fluxes telescope, so particle number is conserved on a
    periodic mesh; and the two operators differ for l_max >= 1."""
    prob = W.periodic_1d(ncells=8, k=2, lmax=3)
    du, dl = dg.Discretisation(prob), dg.Discretisation(_with_flux(prob, "llf"))
    rng = np.random.default_rng(12)
    diff = (dl.D - du.D).toarray()
    for _ in range(20):
        x = rng.standard_normal(du.N)
        assert x @ diff @ x >= -1e-12 * np.abs(diff).max() * (x @ x)
    assert np.abs(diff).max() > 1e-3
    w = np.zeros(dl.N)
    n, nloc = dl.n, dl.mesh.nloc
    for c in range(dl.mesh.ncell):
        w[dl.dof(c, 0, 0): dl.dof(c, 0, 0) + nloc] = 1.0
    Mw = dl.M.T @ w
    colsum = dl.D.T @ w  # sum over the f_000 test functions of every column
    assert np.abs(colsum).max() < 1e-12 * np.abs(dl.D).max(), np.abs(colsum).max()
    assert Mw.any()


@pytest.mark.parametrize("k", [1, 2])
def test_llf_convergence_study_space(k):
    """With the LLF flux the error of the Sec. 4.1 problem against its closed form still falls as
    Delta x^(k+1)."""
    errs = []
    ncs = (8, 16, 32)
    for nc in ncs:
        prob, ex = _convergence_problem(nc, k)
        disc = dg.Discretisation(_with_flux(prob, "llf"))
        z = steppers.rk4(disc.M, disc.D, disc.h, dg.project_initial(disc, prob.f0), 0.005, 200)
        errs.append(_rel_l2_000(disc, z, ex, 1.0, k, nc))
    assert convergence_order(ncs, errs) > k + 1 - 0.3, errs
