"""Field gradients of the library's adjoint step (sap_adjoint_step) against the FP64 oracle.

J = w . zeta_N after N steps (CN and RK4) of a small shock.  The library accumulates dJ/d(field) at
the points where each field is sampled; contracted with a smooth perturbation of that field at the
same points it must equal the oracle's tangent-linear trajectory (steppers.cn_tangent /
steppers.rk4_tangent) along the same perturbation, with dD/deps from the oracle's Richardson
difference of its assembled D (dg.parameter_derivative).  The oracle samples the fields at the same
Gauss points, so one perturbation function serves both.  Directions: U alone (volume and face
points), d U_x/dx alone, DU_x/Dt alone, B_x and B_y, and the shock speed U1 (all of them together,
through the workload's own dependence on U1).  Bound: 1e-7 relative (the Richardson truncation at
step 1e-3 is ~1e-10, the CN solves run to 1e-13)."""
import dataclasses

import numpy as np
import pytest

from paper_2501_05110_gb300 import workloads as W

pytestmark = pytest.mark.gpu

XR, LNPR, NX, NPC, LMAX = (-20.0, 20.0), (0.0, 4.0), 10, 6, 3


def _base(U1=0.1):
    """A small shock with an oblique field B = (0.8, 0.6, 0): the rotation then couples m = 0 to
    m = 1, so every field below changes J (with B along x the m = 0 solution never feels B_x)."""
    p = W.shock(nx=NX, npc=NPC, lmax=LMAX, xr=XR, lnpr=LNPR, U1=U1, Ls=2.0)
    return dataclasses.replace(p, B=lambda xs: np.tile([0.8, 0.6, 0.0], (xs.shape[0], 1)))


def _perturbed(kind, eps):
    """The base problem with one field perturbed by eps times a smooth function of x.  grad U and
    DU/Dt are perturbed relative to their base values: away from the shock the base beta^p is tiny
    (~1e-10), and an absolute perturbation over the Richardson step would carry its eigenvalues
    through zero, where |beta^p| has a kink and a difference quotient no longer approximates the
    derivative."""
    p = _base()
    U, G, DU, B = p.U, p.gradU, p.DUDt, p.B
    if kind == "U":
        def f(xs):
            out = U(xs)
            out[:, 0] += eps * 0.02 * np.cos(0.3 * xs[:, 0])
            return out
        return dataclasses.replace(p, U=f)
    if kind == "gradU":
        def f(xs):
            out = G(xs)
            out[:, 0, 0] *= 1.0 + eps * (1.0 + 0.5 * np.sin(0.2 * xs[:, 0]))
            return out
        return dataclasses.replace(p, gradU=f)
    if kind == "DUDt":
        def f(xs):
            out = DU(xs)
            out[:, 0] *= 1.0 + eps * (1.0 + 0.3 * np.cos(0.1 * xs[:, 0]))
            return out
        return dataclasses.replace(p, DUDt=f)
    if kind == "B":
        def f(xs):
            out = B(xs)
            out[:, 0] += eps * 0.3 * np.sin(0.25 * xs[:, 0])
            out[:, 1] += eps * 0.2 * np.cos(0.15 * xs[:, 0])
            return out
        return dataclasses.replace(p, B=f)
    if kind == "U1":
        return _base(0.1 * (1.0 + eps))
    raise KeyError(kind)


def _direction(sol, kind):
    """The perturbation's derivative d(field)/deps at the library's points (field arrays)."""
    h = 1e-6
    fp = sol.field_arrays(_perturbed(kind, h))
    fm = sol.field_arrays(_perturbed(kind, -h))
    out = {}
    for k in fp:
        if fp[k] is None:
            continue
        d = (fp[k] - fm[k]) / (2 * h)
        if kind == "U1":  # exact: the workload's fields are polynomials in U1
            d = sol.field_arrays(W.shock_U1_derivative(_base(0.1), 0.1))[k] * 0.1
        out[k] = d
    return out


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2501_05110_gb300 import build as sap_build
    sap_build.build()
    return torch


def _library_grads(torch, scheme, dt, nsteps, w):
    from paper_2501_05110_gb300 import sapgpu
    sol = sapgpu.Solver(_base())
    y = sol.initial_state()
    states = [y.clone()]
    for _ in range(nsteps):
        if scheme == "cn":
            sol.step_cn(y, dt, 1, tol=1e-13, restart=30, maxit=4000)
        else:
            sol.step_erk(y, dt, 1)
        states.append(y.clone())
    lam = torch.from_numpy(w).cuda()
    grads = sol.field_grad_buffers()
    for k in range(nsteps, 0, -1):
        sol.adjoint_step(scheme, states[k - 1], states[k] if scheme == "cn" else None, lam, dt, grads, tol=1e-13)
    torch.cuda.synchronize()
    return sol, {k: (None if v is None else v.cpu().numpy()) for k, v in grads.items()}


def _oracle_tangent(kind, scheme, dt, nsteps, w):
    from oracle import dg, steppers
    d0 = dg.Discretisation(_base())
    dD = dg.parameter_derivative(lambda e: _perturbed(kind, e), 0.0, 1e-3)
    if scheme == "cn":
        _, dz = steppers.cn_tangent(d0.M, d0.D, d0.h, dD, np.zeros(d0.N), dt, nsteps)
    else:
        _, dz = steppers.rk4_tangent(d0.M, d0.D, d0.h, dD, np.zeros(d0.N), dt, nsteps)
    return float(w @ d0.to_gauss_nodal(dz))


# RK4: spectral radius of M^-1 D about 320 here (collision up to nu l(l+1)/2 = 6 e^4): dt = 0.004
CASES = {"cn": (1.0, 5), "erk4": (0.004, 6)}


@pytest.fixture(scope="module")
def grads_by_scheme(torch_cuda):
    w = np.random.default_rng(29).standard_normal(_base().ndofs)
    out = {}
    for scheme, (dt, nsteps) in CASES.items():
        sol, g = _library_grads(torch_cuda, scheme, dt, nsteps, w)
        out[scheme] = (sol, g)
    return w, out


@pytest.mark.parametrize("scheme", list(CASES))
@pytest.mark.parametrize("kind", ["U", "gradU", "DUDt", "B", "U1"])
def test_field_gradient_vs_oracle_tangent(grads_by_scheme, scheme, kind):
    w, res = grads_by_scheme
    sol, g = res[scheme]
    dt, nsteps = CASES[scheme]
    d = _direction(sol, kind)
    lib = sum(float(g[k] @ d[k]) for k in d if g.get(k) is not None)
    want = _oracle_tangent(kind, scheme, dt, nsteps, w)
    assert abs(want) > 0
    print(f"field gradient {scheme} {kind}: library {lib:.12e} oracle {want:.12e} rel {abs(lib - want) / abs(want):.2e}")
    assert abs(lib - want) < 1e-7 * abs(want), (lib, want)


def test_field_gradient_source_and_nu(grads_by_scheme):
    """s_000 and nu enter linearly: the library's nodal gradients contracted with a perturbation
    equal the oracle tangent with the exact dD (nu) and the source derivative (s_000: CN adds
    dt mu^T ds, expressed through a second tangent run with dD = 0 and dh)."""
    from oracle import dg, steppers
    import scipy.sparse.linalg as spla
    import scipy.sparse as sp
    w, res = grads_by_scheme
    sol, g = res["cn"]
    dt, nsteps = CASES["cn"]
    rng = np.random.default_rng(31)
    dnu = rng.uniform(0.5, 1.5, g["nu"].size)
    ds = rng.uniform(-1.0, 1.0, g["s000"].size)
    p = _base()
    d0 = dg.Discretisation(p)
    # nu direction: a nodal field (library phase-node order = oracle Gauss points)
    vals = np.ascontiguousarray(dnu)
    pnu = dataclasses.replace(p, nu=lambda xs, pp, _v=vals: _v, terms=frozenset({"coll"}))
    dD = dg.Discretisation(pnu).D
    _, dz = steppers.cn_tangent(d0.M, d0.D, d0.h, dD, np.zeros(d0.N), dt, nsteps)
    want_nu = float(w @ d0.to_gauss_nodal(dz))
    assert abs(float(g["nu"] @ dnu) - want_nu) < 1e-9 * abs(want_nu)
    # source direction: d zeta^n solves (M + dt/2 D) d^n = (M - dt/2 D) d^(n-1) + dt dh
    psrc = dataclasses.replace(p, s000=lambda xs, pp, _v=np.ascontiguousarray(ds): _v)
    dh = dg.Discretisation(psrc).h
    lhs = spla.splu(sp.csc_matrix(d0.M + 0.5 * dt * d0.D))
    rhs = d0.M - 0.5 * dt * d0.D
    dzs = np.zeros(d0.N)
    for _ in range(nsteps):
        dzs = lhs.solve(rhs @ dzs + dt * dh)
    want_s = float(w @ d0.to_gauss_nodal(dzs))
    assert abs(float(g["s000"] @ ds) - want_s) < 1e-9 * abs(want_s)
