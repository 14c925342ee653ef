"""Seeded synthetic problem definitions (inputs only).

This module defines the problems the library is run and checked on: the reduced phase-space
axes, mesh edges, dG degree, expansion order, boundary conditions, active terms and the
prescribed fields U(x), grad U, dU/dt, B (or omega), nu(x,p), the isotropic source s_000 and the
initial condition.  It holds none of the method's arithmetic: no coupling matrices, no quadrature,
no fluxes.  The CUDA binding evaluates these fields at the points the library reports; the CPU
oracle evaluates them at its own quadrature points.

Field call conventions (vectorised over P points):
  U(xs) -> (P,3);  gradU(xs) -> (P,3,3) with [a,b] = dU_b/dx^a;  DUDt(xs) -> (P,3)
  B(xs) -> (P,3) (momentum runs; omega = B / (gamma m));  omega(xs) -> (P,3) (monoenergetic runs)
  nu(xs, p) -> (P,);  s000(xs, p) -> (P,);  f0(coords) -> (P, n)
where ``xs`` holds the resolved spatial coordinates and ``p`` the momentum (not its logarithm) or
None without a momentum axis.  ``coords`` are full phase-space coordinates in axis order.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional, Sequence

import numpy as np

_SPATIAL = ("x", "y", "z")


@dataclasses.dataclass
class Problem:
    name: str
    axes: Sequence[str]                  # e.g. ("x",), ("x", "lnp"), ("x", "y", "z")
    edges: Sequence[np.ndarray]          # per-axis cell edges (graded meshes allowed)
    k: int                               # dG degree
    lmax: int                            # expansion order; n = (lmax+1)^2
    bc: Sequence[tuple]                  # per axis (lo, hi): "periodic" | "inflow0" | "continuous"
    terms: frozenset                     # subset of {"adv", "mom", "rot", "coll", "src"}
    U: Callable
    gradU: Callable
    DUDt: Callable
    nu: Callable
    s000: Callable
    f0: Callable
    B: Optional[Callable] = None         # momentum runs
    omega: Optional[Callable] = None     # monoenergetic runs
    V: float = 1.0                       # monoenergetic particle speed
    dt: float = 1e-3
    nsteps: int = 1
    scheme: str = "erk4"                 # "erk4" | "cn"
    gmres_tol: float = 1e-10
    gmres_restart: int = 30
    flux: str = "upwind"                 # "upwind" (Eq. definition-upwind-flux) | "llf" (local Lax--Friedrichs)

    @property
    def n(self) -> int:
        return (self.lmax + 1) ** 2

    @property
    def ncells(self) -> list:
        return [len(e) - 1 for e in self.edges]

    @property
    def ndofs(self) -> int:
        return int(np.prod(self.ncells)) * self.n * (self.k + 1) ** len(self.axes)

    @property
    def momentum(self) -> Optional[str]:
        m = [a for a in self.axes if a in ("p", "lnp")]
        return m[0] if m else None


def _const3(v):
    v = np.asarray(v, dtype=float)
    return lambda xs: np.broadcast_to(v, (xs.shape[0], 3)).copy()


def _zero33(xs):
    return np.zeros((xs.shape[0], 3, 3))


def _scalar(c):
    return lambda xs, p=None: np.full(xs.shape[0], float(c))


def _iso_f0(fun, n):
    """Initial condition with only f_000 non-zero."""
    def f0(coords):
        out = np.zeros((coords.shape[0], n))
        out[:, 0] = fun(coords)
        return out
    return f0


# ------------------------------------------------------------------------------------------------
# 1-D periodic advection--collision run, ERK4
# ------------------------------------------------------------------------------------------------
def periodic_1d(ncells=64, k=2, lmax=3, U=0.1, nu=1.0, V=1.0, dt=1e-3, nsteps=1000, L=20.0):
    """x in [-L/2, L/2] periodic, constant U along x, B = 0, constant nu, speed V, no momentum
    axis; f_000(x,0) = exp(-x^2/2), other coefficients zero; explicit RK4."""
    n = (lmax + 1) ** 2
    return Problem(
        name=f"periodic1d_x{ncells}_k{k}_l{lmax}",
        axes=("x",), edges=[np.linspace(-L / 2, L / 2, ncells + 1)], k=k, lmax=lmax,
        bc=[("periodic", "periodic")], terms=frozenset({"adv", "rot", "coll"}),
        U=_const3([U, 0, 0]), gradU=_zero33, DUDt=_const3([0, 0, 0]),
        omega=_const3([0, 0, 0]), V=V, nu=_scalar(nu), s000=_scalar(0.0),
        f0=_iso_f0(lambda c: np.exp(-0.5 * c[:, 0] ** 2), n),
        dt=dt, nsteps=nsteps, scheme="erk4")


# ------------------------------------------------------------------------------------------------
# parallel shock in (x, ln p), Crank--Nicolson
# ------------------------------------------------------------------------------------------------
def shock_profile(U1, r, Ls):
    """U(x) = U1 [(1+1/r)/2 - (1-1/r)/2 tanh(x/Ls)] along x, its gradient and (U.grad)U."""
    a, b = 0.5 * (1 + 1 / r), 0.5 * (1 - 1 / r)

    def U(xs):
        out = np.zeros((xs.shape[0], 3))
        out[:, 0] = U1 * (a - b * np.tanh(xs[:, 0] / Ls))
        return out

    def dUdx(x):
        e = np.exp(-2.0 * np.abs(x) / Ls)  # sech^2(y) = 4 e^{-2|y|} / (1 + e^{-2|y|})^2
        return -U1 * b / Ls * 4.0 * e / (1.0 + e) ** 2

    def gradU(xs):
        out = np.zeros((xs.shape[0], 3, 3))
        out[:, 0, 0] = dUdx(xs[:, 0])
        return out

    def DUDt(xs):
        out = np.zeros((xs.shape[0], 3))
        out[:, 0] = U(xs)[:, 0] * dUdx(xs[:, 0])
        return out

    return U, gradU, DUDt


def shock(nx=256, npc=64, k=1, lmax=3, U1=0.1, r=4.0, Ls=0.5, xr=(-200.0, 200.0), lnpr=(0.0, 10.0),
          nu0=1.0, nu_field=None, Q=0.1, x0=0.0, lnp0=1.0, sig_x=None, sig_lnp=None, B0=1.0,
          dt=1.0, nsteps=2000, tol=1e-10, restart=30, x_edges=None, name=None, momentum="lnp"):
    """Parallel shock (Sec. 4.4 set-up, with this library's readings of its open points): x upstream
    zero inflow, x downstream continuous, ln p zero inflow at both ends; nu = nu0 p (or a given
    field); B = B0 e_x; Gaussian isotropic source at (x0, ln p0) with rate Q; zero initial state;
    Crank--Nicolson with GMRES.  momentum="p" resolves linear p instead of ln p: the momentum axis
    then has uniform cells in p over [exp(lnpr[0]), exp(lnpr[1])] (the source keeps its ln p shape)."""
    xe = np.linspace(xr[0], xr[1], nx + 1) if x_edges is None else np.asarray(x_edges, float)
    if momentum == "p":
        pe = np.linspace(math.exp(lnpr[0]), math.exp(lnpr[1]), npc + 1)
    else:
        pe = np.linspace(lnpr[0], lnpr[1], npc + 1)
    dx = (xe[-1] - xe[0]) / (len(xe) - 1)
    dlnp = (lnpr[1] - lnpr[0]) / npc
    sx = 2 * dx if sig_x is None else sig_x
    sp_ = 2 * dlnp if sig_lnp is None else sig_lnp
    n = (lmax + 1) ** 2
    U, gradU, DUDt = shock_profile(U1, r, Ls)
    nu = nu_field if nu_field is not None else (lambda xs, p: nu0 * np.asarray(p, float))

    def s000(xs, p):
        s = Q / (2 * math.pi * sx * sp_) * np.exp(-(xs[:, 0] - x0) ** 2 / (2 * sx ** 2)) \
            * np.exp(-(np.log(p) - lnp0) ** 2 / (2 * sp_ ** 2))
        return math.sqrt(4 * math.pi) * s

    return Problem(
        name=name or f"shock_x{len(xe)-1}_{momentum}{npc}_k{k}_l{lmax}",
        axes=("x", momentum), edges=[xe, pe], k=k, lmax=lmax,
        bc=[("inflow0", "continuous"), ("inflow0", "inflow0")],
        terms=frozenset({"adv", "mom", "rot", "coll", "src"}),
        U=U, gradU=gradU, DUDt=DUDt, B=_const3([B0, 0, 0]), nu=nu, s000=s000,
        f0=lambda c: np.zeros((c.shape[0], n)),
        dt=dt, nsteps=nsteps, scheme="cn", gmres_tol=tol, gmres_restart=restart)


def shock_U1_derivative(prob, U1):
    """d/dU1 of the shock's prescribed fields, as a Problem with the same points: U and grad U are
    linear in U1 and (U.grad)U is quadratic (see shock_profile), so dU/dU1 = U/U1,
    d(grad U)/dU1 = grad U / U1, d(DU/Dt)/dU1 = 2 (DU/Dt) / U1; B, nu and the source do not depend
    on U1."""
    U, G, DU = prob.U, prob.gradU, prob.DUDt
    zero = lambda xs, p=None: np.zeros(xs.shape[0])
    return dataclasses.replace(
        prob, U=lambda xs: U(xs) / U1, gradU=lambda xs: G(xs) / U1, DUDt=lambda xs: 2.0 * DU(xs) / U1,
        B=_const3([0, 0, 0]), omega=_const3([0, 0, 0]), nu=zero, s000=zero)


# ------------------------------------------------------------------------------------------------
# 3-D periodic box with oblique field, ERK4
# ------------------------------------------------------------------------------------------------
def box3d(ncells=48, k=2, lmax=5, nu=0.5, L=20.0, V=1.0, dt=0.01, nsteps=200, seed=3, nbumps=8, sigma=1.5):
    """Periodic box [-L/2, L/2]^3, U = 0, omega = (cos 45, sin 45, 0), constant nu, speed V;
    f_000 = 1 + 0.5 sum_b a_b exp(-|x - c_b|_per^2 / (2 sigma^2)) with seeded centres and
    amplitudes (random-phase Gaussian bumps), other coefficients zero; explicit RK4."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-L / 2, L / 2, size=(nbumps, 3))
    amps = rng.uniform(0.5, 1.0, size=nbumps)
    n = (lmax + 1) ** 2

    def f000(c):
        out = np.ones(c.shape[0])
        for cb, ab in zip(centres, amps):
            d = c[:, :3] - cb
            d -= L * np.round(d / L)
            out += 0.5 * ab * np.exp(-np.sum(d * d, axis=1) / (2 * sigma ** 2))
        return out

    e = np.linspace(-L / 2, L / 2, ncells + 1)
    c45 = math.cos(math.pi / 4)
    return Problem(
        name=f"box3d_{ncells}c_k{k}_l{lmax}",
        axes=("x", "y", "z"), edges=[e, e.copy(), e.copy()], k=k, lmax=lmax,
        bc=[("periodic", "periodic")] * 3, terms=frozenset({"adv", "rot", "coll"}),
        U=_const3([0, 0, 0]), gradU=_zero33, DUDt=_const3([0, 0, 0]),
        omega=_const3([c45, c45, 0.0]), V=V, nu=_scalar(nu), s000=_scalar(0.0),
        f0=_iso_f0(f000, n), dt=dt, nsteps=nsteps, scheme="erk4")


# ------------------------------------------------------------------------------------------------
# advection in a constant magnetic field (gyration), ERK4
# ------------------------------------------------------------------------------------------------
def gyro_advection(ncells=64, k=3, lmax=3, U0=0.1, L=20.0, gamma=2.0, B0=2.0 * math.pi, sigma=1.5, dt=0.02,
                   nsteps=10000):
    """Monoenergetic particles in a constant field B = B0 e_z without scattering, in a periodic
    (x, y) box of side L moving with U = (U0, U0, 0) (U0 = 0: static plasma); f_000 = Gaussian of
    width sigma, other coefficients zero (Sec. 4.2 set-up).  omega = B0 / gamma, V = sqrt(1 - 1/gamma^2);
    the distribution returns to its initial state after N gyro-periods when L = N U0 T_g."""
    n = (lmax + 1) ** 2
    omega = B0 / gamma
    V = math.sqrt(1.0 - 1.0 / gamma ** 2)
    e = np.linspace(-L / 2, L / 2, ncells + 1)
    return Problem(
        name=f"gyro_{ncells}c_k{k}_l{lmax}_U{U0}",
        axes=("x", "y"), edges=[e, e.copy()], k=k, lmax=lmax,
        bc=[("periodic", "periodic")] * 2, terms=frozenset({"adv", "rot"}),
        U=_const3([U0, U0, 0]), gradU=_zero33, DUDt=_const3([0, 0, 0]),
        omega=_const3([0, 0, omega]), V=V, nu=_scalar(0.0), s000=_scalar(0.0),
        f0=_iso_f0(lambda c: np.exp(-(c[:, 0] ** 2 + c[:, 1] ** 2) / (2 * sigma ** 2)), n),
        dt=dt, nsteps=nsteps, scheme="erk4")


# ------------------------------------------------------------------------------------------------
# closure: free streaming of an initially isotropic Gaussian, ERK4
# ------------------------------------------------------------------------------------------------
def closure(ncells=256, k=2, lmax=11, nu=0.0, gamma=2.0, sigma=1.0, xr=(-15.0, 15.0), dt=None, nsteps=None):
    """Monoenergetic particles streaming along x with scattering rate nu (Sec. 4.3 set-up): 1-D,
    terms spatial advection and collision, f_000(x, 0) = sqrt(2)/sigma exp(-x^2/(2 sigma^2)) (the
    Y_000 projection of an isotropic Gaussian of unit mass), zero-inflow boundaries far from the
    particles; dt = 1/(100 sqrt(3)) and t_F = 12/sqrt(3) by default."""
    n = (lmax + 1) ** 2
    V = math.sqrt(1.0 - 1.0 / gamma ** 2)
    dt = 1.0 / (100.0 * math.sqrt(3.0)) if dt is None else dt
    nsteps = int(round((12.0 / math.sqrt(3.0)) / dt)) if nsteps is None else nsteps
    return Problem(
        name=f"closure_{ncells}c_k{k}_l{lmax}_nu{nu}",
        axes=("x",), edges=[np.linspace(xr[0], xr[1], ncells + 1)], k=k, lmax=lmax,
        bc=[("inflow0", "inflow0")], terms=frozenset({"adv", "coll"}),
        U=_const3([0, 0, 0]), gradU=_zero33, DUDt=_const3([0, 0, 0]),
        omega=_const3([0, 0, 0]), V=V, nu=_scalar(nu), s000=_scalar(0.0),
        f0=_iso_f0(lambda c: math.sqrt(2.0) / sigma * np.exp(-c[:, 0] ** 2 / (2 * sigma ** 2)), n),
        dt=dt, nsteps=nsteps, scheme="erk4")


# ------------------------------------------------------------------------------------------------
# diffusive shock acceleration at a parallel shock (the paper's production set-up)
# ------------------------------------------------------------------------------------------------
def dsa_x_edges(Ls=1.0 / 25.0, dx_shock=0.01, growth=0.01, xmax=280.0):
    """Cells of width dx_shock across the shock region [-Ls, Ls], then widths sinh(growth i),
    i = 1, 2, ..., on both sides until |x| = xmax (the last cell ends at xmax)."""
    inner = np.linspace(-Ls, Ls, int(round(2 * Ls / dx_shock)) + 1)
    right = [Ls]
    i = 1
    while right[-1] < xmax:
        right.append(min(right[-1] + math.sinh(growth * i), xmax))
        i += 1
    if right[-1] - right[-2] < 0.5 * math.sinh(growth * (i - 2)):  # merge a sliver into its neighbour
        del right[-2]
    right = np.array(right[1:])
    return np.concatenate([-right[::-1], inner, right])


def dsa_shock(npc=256, k=1, p0=2.0, Q=0.1, dt=1.0, nsteps=500000):
    """Diffusive shock acceleration (Sec. 4.4, Tab. of simulation parameters): l_max = 1, U1 = 1/60,
    r = 4, L_s = 1/25, nu = 1, B0 = 1, injection at x0 = 0 and p0 = 2 with widths 1/8 in x and in p,
    domain [-280, 280] x [ln 0.1, ln 100] with 256 ln p cells, graded x-cells (dsa_x_edges), CN with
    dt = 1.  The paper injects Q particles per unit time at p0 (per unit p); the shock workload's
    source is a Gaussian per unit ln p, so it carries Q / p0 with width (1/8) / p0 in ln p."""
    return shock(x_edges=dsa_x_edges(), npc=npc, k=k, lmax=1, U1=1.0 / 60.0, r=4.0, Ls=1.0 / 25.0,
                 lnpr=(math.log(0.1), math.log(100.0)), nu_field=lambda xs, p: np.ones(xs.shape[0]),
                 Q=Q / p0, x0=0.0, lnp0=math.log(p0), sig_x=0.125, sig_lnp=0.125 / p0, B0=1.0, dt=dt,
                 nsteps=nsteps, name="dsa_shock")


def dsa_phi(t, c1=78909.74, sd=48859.1):
    """Approximate time dependence of the spectrum at the shock, phi(t) = int_0^t zeta (Sec. 4.4,
    Eq. cumulative-temporal-distribution), with the mean c1 and standard deviation of the
    acceleration time the paper gives for p = 59.9."""
    from math import erfc, exp, sqrt
    c2 = sd * sd
    a = sqrt(c1 ** 3 / (2.0 * t * c2))
    b = sqrt(c1 * t / (2.0 * c2))
    return 0.5 * (exp(2.0 * c1 * c1 / c2) * erfc(a + b) + erfc(a - b))


# ------------------------------------------------------------------------------------------------
# batched shocks
# ------------------------------------------------------------------------------------------------
def batched_shocks(count=512, seed=4, npc=64, nx_range=(64, 512), lmax_choices=(1, 3, 5, 7), **kw):
    """Independent shock instances: r ~ U[2,4], log nu0 ~ U[log 0.1, log 10], lmax uniform over
    ``lmax_choices``, x-cell count uniform over nx_range (inclusive); otherwise as ``shock``."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        r = rng.uniform(2.0, 4.0)
        nu0 = math.exp(rng.uniform(math.log(0.1), math.log(10.0)))
        lmax = int(rng.choice(lmax_choices))
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        out.append(shock(nx=nx, npc=npc, lmax=lmax, r=r, nu0=nu0, name=f"batch{i}", **kw))
    return out


# ------------------------------------------------------------------------------------------------
# per-cell scattering field for the adjoint run
# ------------------------------------------------------------------------------------------------
def lognormal_cell_nu(x_edges, lnp_edges, sigma=0.3, seed=6):
    """nu_c = p_c exp(sigma z_c), z_c ~ N(0,1) per cell, p_c = exp(cell-centre ln p);
    returns (nu(xs, p), z) with z of shape (npc, nx)."""
    rng = np.random.default_rng(seed)
    nx, npc = len(x_edges) - 1, len(lnp_edges) - 1
    z = rng.standard_normal((npc, nx))
    pc = np.exp(0.5 * (lnp_edges[:-1] + lnp_edges[1:]))

    def nu(xs, p):
        ix = np.clip(np.searchsorted(x_edges, xs[:, 0], side="right") - 1, 0, nx - 1)
        ip = np.clip(np.searchsorted(lnp_edges, np.log(p), side="right") - 1, 0, npc - 1)
        return pc[ip] * np.exp(sigma * z[ip, ix])

    return nu, z


# ------------------------------------------------------------------------------------------------
# named workloads
# ------------------------------------------------------------------------------------------------
def config(name: str) -> Problem:
    if name == "periodic1d":
        return periodic_1d()
    if name == "shock":
        return shock()
    if name == "box3d":
        return box3d()
    raise KeyError(name)
