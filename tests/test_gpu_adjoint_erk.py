"""Discrete adjoint of RK4 trajectories (library adjoint step + torch.autograd.Function with
checkpoints): one step against the oracle's transposed RK4 step, gradients with respect to a per-cell
nu(x, p) against the oracle's tangent-linear RK4 trajectory, and the U1 gradient (library field
gradients chained to U1) against central finite differences of GPU trajectories and the oracle's
tangent."""
import numpy as np
import pytest

from paper_2501_05110_gb300 import workloads as W

from .oracle_bridge import NodalOracle

pytestmark = pytest.mark.gpu

XR, LNPR, NX, NPC, LMAX = (-20.0, 20.0), (0.0, 4.0), 10, 6, 3
DT, NSTEPS = 0.004, 6  # spectral radius of M^-1 D is 319 here: RK4 is stable for dt < 0.0087


def _base(U1, nu_field=None):
    return W.shock(nx=NX, npc=NPC, lmax=LMAX, xr=XR, lnpr=LNPR, U1=U1, nu_field=nu_field)


@pytest.fixture(scope="module")
def setup():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2501_05110_gb300 import build as sap_build
    sap_build.build()
    from paper_2501_05110_gb300 import adjoint, sapgpu
    prob0 = _base(0.1)
    xe, pe = prob0.edges
    nu_cell_fun, _ = W.lognormal_cell_nu(xe, pe, seed=6)
    probe = sapgpu.Solver(_base(0.1, nu_cell_fun))
    pts = probe.points(sapgpu.PTS_PHASE)
    nu_nodes = nu_cell_fun(pts[:, :1], np.exp(pts[:, 1]))
    probe.close()

    def make(nu_np, U1):
        vals = np.ascontiguousarray(nu_np if nu_np is not None else nu_nodes, dtype=np.float64)
        return _base(U1, lambda xs_, p_, _v=vals: _v)

    w = torch.from_numpy(np.random.default_rng(17).standard_normal(prob0.ndofs)).cuda()
    return dict(torch=torch, adjoint=adjoint, sapgpu=sapgpu, nu_nodes=nu_nodes, make=make, w=w,
                nu_cell_fun=nu_cell_fun, edges=(xe, pe), cell_of_node=np.arange(len(nu_nodes)) // 4)


def _J_forward(S, nu_np, U1):
    sol = S["sapgpu"].Solver(S["make"](nu_np, U1))
    y = sol.initial_state()
    sol.step_erk(y, DT, NSTEPS)
    S["torch"].cuda.synchronize()
    val = float(S["w"] @ y)
    sol.close()
    return val


def _adjoint_grads(S, checkpoint):
    torch = S["torch"]
    fam = S["adjoint"].CNProblemFamily(make_problem=S["make"], nsteps=NSTEPS, dt=DT, checkpoint=checkpoint)
    nu_t = torch.tensor(S["nu_nodes"], dtype=torch.float64, device="cuda", requires_grad=True)
    u1_t = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
    zN = S["adjoint"].ERKTrajectory.apply(nu_t, u1_t, fam)
    J = (S["w"] * zN).sum()
    J.backward()
    g_node = nu_t.grad.cpu().numpy()
    return np.bincount(S["cell_of_node"], weights=g_node), float(u1_t.grad), float(J.detach())


@pytest.mark.parametrize("name", ["shock_small", "box_tiny", "box_k2_node", "periodic1d_tiny"])
def test_adjoint_erk_step_vs_oracle_transpose(setup, name):
    """One library RK4 adjoint step equals the oracle's transposed RK4 step (stability polynomial
    in the transposed nodal operator, built column by column from the oracle), element by element."""
    torch = setup["torch"]
    sapgpu = setup["sapgpu"]
    prob = {"shock_small": lambda: W.shock(nx=4, npc=3, lmax=2, xr=(-4.0, 4.0), lnpr=(0.0, 2.0)),
            "box_tiny": lambda: W.box3d(ncells=2, k=1, lmax=2),
            # k = 2: the forward stages run the node kernel, the transposed ones the row kernel
            "box_k2_node": lambda: W.box3d(ncells=2, k=2, lmax=2),
            "periodic1d_tiny": lambda: W.periodic_1d(ncells=5, k=2, lmax=2)}[name]()
    from oracle import steppers
    orc = NodalOracle(prob)
    sol = sapgpu.Solver(prob)
    N = sol.N
    eye = np.eye(N)
    O = np.stack([orc.apply(eye[:, j]) for j in range(N)], axis=1)  # nodal M^-1 D
    rho = np.abs(np.linalg.eigvals(O)).max()
    dt = 1.0 / rho
    rng = np.random.default_rng(5)
    y, lam = rng.standard_normal(N), rng.standard_normal(N)
    want = steppers.rk4_step_transpose(lambda x: O.T @ x, dt, lam)
    lam_t = torch.from_numpy(lam).cuda()
    st = sol.adjoint_step_erk(torch.from_numpy(y).cuda(), lam_t, dt)
    torch.cuda.synchronize()
    got = lam_t.cpu().numpy()
    sol.close()
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
    assert st.kernel_launches >= 8


def test_adjoint_erk_J_and_checkpoint_invariance(setup):
    """The autograd trajectory reproduces the plain forward J, and the gradients do not depend on
    the checkpoint interval (RK4 recomputation repeats the forward states exactly)."""
    S = setup
    a = _adjoint_grads(S, checkpoint=1)
    b = _adjoint_grads(S, checkpoint=50)
    assert abs(a[2] - _J_forward(S, None, 0.1)) <= 1e-14 * abs(a[2])
    assert np.allclose(a[0], b[0], rtol=1e-13, atol=1e-15 * np.abs(a[0]).max())
    assert abs(a[1] - b[1]) <= 1e-12 * abs(a[1])


def test_adjoint_erk_nu_gradient_vs_oracle_tangent(setup):
    """Directional derivative along a random per-cell direction: adjoint gradient . v equals the FP64
    oracle's tangent-linear RK4 trajectory, contracted with the same weights (nodal basis)."""
    from oracle import dg, steppers
    S = setup
    xe, pe = S["edges"]
    g_cell, _, _ = _adjoint_grads(S, checkpoint=2)
    v = np.random.default_rng(23).standard_normal((len(pe) - 1, len(xe) - 1))

    def cellfun(vals):
        def f(xs, p):
            ix = np.clip(np.searchsorted(xe, xs[:, 0], side="right") - 1, 0, len(xe) - 2)
            ip = np.clip(np.searchsorted(pe, np.log(p), side="right") - 1, 0, len(pe) - 2)
            return vals[ip, ix]
        return f

    d0 = dg.Discretisation(_base(0.1, S["nu_cell_fun"]))
    pv = _base(0.1, cellfun(v))
    pv.terms = frozenset({"coll"})
    dD = dg.Discretisation(pv).D
    _, dz = steppers.rk4_tangent(d0.M, d0.D, d0.h, dD, np.zeros(d0.N), DT, NSTEPS)
    dJ_oracle = float(S["w"].cpu().numpy() @ d0.to_gauss_nodal(dz))
    dJ_adj = float(np.sum(g_cell * v.reshape(-1)))  # cells: x fastest, as v.reshape
    assert abs(dJ_adj - dJ_oracle) < 1e-8 * abs(dJ_oracle), (dJ_adj, dJ_oracle)


def test_adjoint_erk_U1_gradient_vs_finite_differences(setup):
    S = setup
    _, g_u1, _ = _adjoint_grads(S, checkpoint=3)
    e = 1e-5 * 0.1
    fd = (_J_forward(S, None, 0.1 + e) - _J_forward(S, None, 0.1 - e)) / (2 * e)
    assert abs(fd - g_u1) < 1e-5 * abs(fd), (fd, g_u1)


def test_adjoint_erk_U1_gradient_vs_oracle_tangent(setup):
    """dJ/dU1 from the library's field gradients equals the FP64 oracle's tangent-linear RK4
    trajectory with dD/dU1 from the Richardson difference of its assembled D."""
    from oracle import dg, steppers
    S = setup
    _, g_u1, _ = _adjoint_grads(S, checkpoint=2)
    make = lambda U1: _base(U1, S["nu_cell_fun"])
    d0 = dg.Discretisation(make(0.1))
    dD = dg.parameter_derivative(make, 0.1, 1e-4)
    _, dz = steppers.rk4_tangent(d0.M, d0.D, d0.h, dD, np.zeros(d0.N), DT, NSTEPS)
    want = float(S["w"].cpu().numpy() @ d0.to_gauss_nodal(dz))
    assert abs(g_u1 - want) < 1e-7 * abs(want), (g_u1, want)


def test_adjoint_steps_degenerate_inputs(setup):
    """lambda = 0: the CN adjoint solve has a zero right side (mu = 0 without iterating) and both
    steps return lambda = 0 and leave the nu-gradient unchanged; dt = 0: the RK4 step is the
    identity, so its adjoint returns lambda unchanged."""
    torch = setup["torch"]
    sol = setup["sapgpu"].Solver(setup["make"](None, 0.1))
    N = sol.N
    g = torch.Generator(device="cuda").manual_seed(9)
    zp = torch.randn(N, device="cuda", dtype=torch.float64, generator=g)
    zn = torch.randn(N, device="cuda", dtype=torch.float64, generator=g)
    grad = torch.randn(len(setup["nu_nodes"]), device="cuda", dtype=torch.float64, generator=g)
    grad0 = grad.clone()
    lam = torch.zeros(N, device="cuda", dtype=torch.float64)
    mu = torch.full((N,), 7.0, device="cuda", dtype=torch.float64)
    st = sol.adjoint_step_cn(zp, zn, lam, 1.0, 1e-12, 30, 100, mu_out=mu, grad_nu=grad)
    assert st.iterations == 0 and not lam.any() and not mu.any()
    sol.adjoint_step_erk(zp, lam, DT, grad_nu=grad)
    torch.cuda.synchronize()
    assert not lam.any() and torch.equal(grad, grad0)
    lam1 = torch.randn(N, device="cuda", dtype=torch.float64, generator=g)
    lam2 = lam1.clone()
    sol.adjoint_step_erk(zp, lam2, 0.0)
    torch.cuda.synchronize()
    assert torch.equal(lam1, lam2)
    sol.close()
