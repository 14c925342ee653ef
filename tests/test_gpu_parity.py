"""Parity of the CUDA library (through the C ABI) with the FP64 CPU oracle.

Tolerances (FP64 path): the operator apply agrees to 1e-12 relative to the largest output entry
(the paper-level bound for the plain path is rel. L2 <= 1e-12); ERK and exactly solved CN
trajectories to 1e-12 relative L2.  Inputs are seeded; sizes span several thread blocks with a
ragged tail.
"""
import numpy as np
import pytest

from paper_2501_05110_gb300 import workloads as W

from .oracle_bridge import NodalOracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2501_05110_gb300 import build as sap_build
    sap_build.build()
    return torch


def _solver(prob, prec="fp64"):
    from paper_2501_05110_gb300 import sapgpu
    return sapgpu.Solver(prob, prec)


def _gpu_apply(torch, solver, y_np, rhs=False, dtype=None):
    from paper_2501_05110_gb300 import sapgpu
    dtype = dtype or torch.float64
    x = torch.from_numpy(y_np).to("cuda", dtype)
    out = torch.empty_like(x)
    solver.apply(x, out, sapgpu.APPLY_RHS if rhs else sapgpu.APPLY_D)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


def _rel_max(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _tiny_problems():
    return [
        W.periodic_1d(ncells=3, k=2, lmax=1),
        W.periodic_1d(ncells=1, k=1, lmax=2),
        W.shock(nx=3, npc=2, lmax=1, xr=(-2.0, 2.0), lnpr=(0.0, 2.0)),
        W.shock(nx=2, npc=3, lmax=2, k=2, xr=(-1.0, 1.0), lnpr=(0.5, 2.0)),
        W.box3d(ncells=2, k=1, lmax=1),
    ]


@pytest.mark.parametrize("idx", range(5))
def test_apply_unit_vectors_tiny(torch_cuda, idx):
    """Brute force on 1-8 cells: every column of M^-1 D matches the oracle's assembled operator."""
    prob = _tiny_problems()[idx]
    orc = NodalOracle(prob)
    sol = _solver(prob)
    N = sol.N
    assert N == orc.disc.N
    eye = np.eye(N)
    G = np.stack([_gpu_apply(torch_cuda, sol, eye[:, j]) for j in range(N)], axis=1)
    O = np.stack([orc.apply(eye[:, j]) for j in range(N)], axis=1)
    assert _rel_max(G, O) < 1e-12


@pytest.mark.parametrize("name", ["periodic1d", "shock_small", "box_small", "shock_graded"])
def test_apply_random(torch_cuda, name):
    rng = np.random.default_rng(11)
    if name == "periodic1d":
        prob = W.periodic_1d()
    elif name == "shock_small":
        prob = W.shock(nx=15, npc=7, lmax=3)
    elif name == "box_small":
        prob = W.box3d(ncells=3, k=2, lmax=3)
    else:
        xe = np.concatenate([-np.geomspace(30, 0.05, 9), np.linspace(-0.04, 0.04, 5), np.geomspace(0.05, 60, 10)])
        prob = W.shock(x_edges=np.sort(xe), npc=6, lmax=2, lnpr=(-1.0, 4.0), Ls=0.05)
    orc = NodalOracle(prob)
    sol = _solver(prob)
    y = rng.standard_normal(sol.N)
    for rhs in (False, True):
        assert _rel_max(_gpu_apply(torch_cuda, sol, y, rhs), orc.apply(y, rhs)) < 1e-12


def test_erk_periodic_1d_full(torch_cuda):
    """RK4, dt = 1e-3, 1000 steps on the 1-D periodic workload; conservation of int f_000 dx."""
    prob = W.periodic_1d()
    orc = NodalOracle(prob)
    sol = _solver(prob)
    y0 = sol.initial_state()
    want = orc.rk4(y0.cpu().numpy(), prob.dt, prob.nsteps)
    y = y0.clone()
    sol.step_erk(y, prob.dt, prob.nsteps)
    torch_cuda.cuda.synchronize()
    got = y.cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12
    # particle number: sum over cells of h * sum_nodes w_node f_000
    w = orc.disc.wg * (20.0 / 64)
    m0 = (y0.cpu().numpy().reshape(64, prob.n, 3)[:, 0, :] * w).sum()
    m1 = (got.reshape(64, prob.n, 3)[:, 0, :] * w).sum()
    assert abs(m1 - m0) < 1e-12 * abs(m0)


def test_cn_shock_small_exact(torch_cuda):
    """CN steps solved to 1e-14 agree with the oracle's sparse-LU CN to 1e-12 (rel. L2)."""
    prob = W.shock(nx=15, npc=7, lmax=3)
    orc = NodalOracle(prob)
    sol = _solver(prob)
    y = sol.initial_state()
    st = sol.step_cn(y, 1.0, 12, tol=1e-14, restart=30, maxit=3000)
    torch_cuda.cuda.synchronize()
    want = orc.cn(np.zeros(sol.N), 1.0, 12)
    got = y.cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12
    assert st.last_rel_residual <= 1e-14 and st.iterations > 0


def test_cn_tolerance_1e10(torch_cuda):
    """At the workload tolerance 1e-10 the CN trajectory stays within steps * tol * cond of LU."""
    prob = W.shock(nx=15, npc=7, lmax=3)
    orc = NodalOracle(prob)
    sol = _solver(prob)
    y = sol.initial_state()
    st = sol.step_cn(y, 1.0, 12, tol=1e-10)
    torch_cuda.cuda.synchronize()
    want = orc.cn(np.zeros(sol.N), 1.0, 12)
    err = np.linalg.norm(y.cpu().numpy() - want) / np.linalg.norm(want)
    assert err < 1e-8 and st.last_rel_residual <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cn_changing_dt_and_fields(torch_cuda, prec):
    """CN calls with changing dt, and after new fields, match the oracle's LU CN run with the same
    sequence: the iteration groups that the library replays from cached CUDA graphs are rebuilt
    whenever dt or the fields change."""
    prob = W.shock(nx=15, npc=7, lmax=3)
    prob2 = W.shock(nx=15, npc=7, lmax=3, nu0=2.0)
    sol = _solver(prob, prec)
    y = sol.initial_state()
    z = np.zeros(sol.N)
    for dt, nsteps in [(1.0, 3), (0.5, 3), (1.0, 2)]:
        sol.step_cn(y, dt, nsteps, tol=1e-13, restart=30, maxit=4000)
        z = NodalOracle(prob).cn(z, dt, nsteps)
    sol.set_fields(prob2)
    sol.step_cn(y, 1.0, 3, tol=1e-13, restart=30, maxit=4000)
    torch_cuda.cuda.synchronize()
    want = NodalOracle(prob2).cn(z, 1.0, 3)
    err = np.linalg.norm(y.cpu().numpy() - want) / np.linalg.norm(want)
    assert err < (1e-11 if prec == "fp64" else 1e-8), err


# ------------------------------------------------------------------------------------------------
# precision form: FP32 operator apply (FP64 state in RK4)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["periodic1d", "shock_small", "box_small"])
def test_apply_fp32(torch_cuda, name):
    """FP32 apply vs the FP64 oracle: error below 1e-5 of the largest output entry."""
    rng = np.random.default_rng(12)
    prob = {"periodic1d": W.periodic_1d(), "shock_small": W.shock(nx=15, npc=7, lmax=3),
            "box_small": W.box3d(ncells=3, k=2, lmax=3)}[name]
    orc = NodalOracle(prob)
    sol = _solver(prob, "fp32")
    y = rng.standard_normal(sol.N)
    got = _gpu_apply(torch_cuda, sol, y, dtype=torch_cuda.float32)
    assert _rel_max(got, orc.apply(y)) < 1e-5


def test_erk_fp32_periodic_1d(torch_cuda):
    """RK4 with FP32 stage derivatives and FP64 accumulation (1000 steps): rel. L2 error vs the
    FP64 oracle below 1e-5 (~1e-6 expected from the FP32 stage derivatives)."""
    prob = W.periodic_1d()
    orc = NodalOracle(prob)
    sol = _solver(prob, "fp32")
    y0 = sol.initial_state()
    want = orc.rk4(y0.cpu().numpy(), prob.dt, prob.nsteps)
    y = y0.clone()
    sol.step_erk(y, prob.dt, prob.nsteps)
    torch_cuda.cuda.synchronize()
    err = np.linalg.norm(y.cpu().numpy() - want) / np.linalg.norm(want)
    assert err < 1e-5, err


# ------------------------------------------------------------------------------------------------
# full-size workloads: sampled outputs and properties
# ------------------------------------------------------------------------------------------------
def _sample_cells(ncell, count, seed):
    rng = np.random.default_rng(seed)
    c = set(rng.choice(ncell, size=count, replace=False).tolist())
    c.update([0, ncell - 1])
    return np.array(sorted(c))


def test_apply_full_shock_sampled(torch_cuda):
    """Full 256 x 64 shock workload: GPU apply on a random state vs the oracle's rows of sampled
    cells (the oracle assembles only those rows)."""
    prob = W.shock()
    sol = _solver(prob)
    y = np.random.default_rng(5).standard_normal(sol.N)
    got = _gpu_apply(torch_cuda, sol, y)
    cells = _sample_cells(256 * 64, 40, 1)
    orc = NodalOracle(prob, rows_of_cells=cells)
    want = orc.apply(y)
    m = orc.row_mask()
    assert _rel_max(got[m], want[m]) < 1e-12


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_apply_full_box3d_sampled(torch_cuda, prec, tol):
    """Full 48^3, k = 2, lmax = 5 box (107.5 M DoFs): sampled cells vs the oracle's rows."""
    import torch
    prob = W.box3d()
    sol = _solver(prob, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    g = torch.Generator(device="cuda").manual_seed(3)
    x = torch.randn(sol.N, device="cuda", dtype=torch.float64, generator=g).to(dt)
    yv = torch.empty_like(x)
    from paper_2501_05110_gb300 import sapgpu
    sol.apply(x, yv, sapgpu.APPLY_D)
    torch.cuda.synchronize()
    cells = _sample_cells(48 ** 3, 40, 2)
    per = prob.n * 27
    idx = torch.from_numpy(np.concatenate([c * per + np.arange(per) for c in cells])).cuda()
    # the oracle needs the input of the sampled cells and of their neighbours: take it all on host
    xin = x.double().cpu().numpy()
    orc = NodalOracle(prob, rows_of_cells=cells)
    want = orc.apply(xin)
    got = yv.double()[idx].cpu().numpy()
    m = orc.row_mask()
    assert _rel_max(got, want[m]) < tol


def test_erk_full_box3d_conservation(torch_cuda):
    """Full 48^3 box, 5 RK4 steps of dt = 0.01 (FP64): int f_000 d^3x is conserved to rounding
    (periodic, U = 0, C_00 = 0, Omega row 0 = 0) and the state stays finite."""
    import torch
    prob = W.box3d()
    sol = _solver(prob)
    y = sol.initial_state()
    w1 = torch.tensor(np.polynomial.legendre.leggauss(3)[1] / 2, device="cuda", dtype=torch.float64)
    w3 = (w1[:, None, None] * w1[None, :, None] * w1[None, None, :]).reshape(-1)
    def mass(v):
        return float((v.view(-1, prob.n, 27)[:, 0, :] * w3).sum())
    m0 = mass(y)
    sol.step_erk(y, prob.dt, 5)
    torch.cuda.synchronize()
    m1 = mass(y)
    assert torch.isfinite(y).all()
    assert abs(m1 - m0) < 1e-12 * abs(m0), (m0, m1)


@pytest.mark.parametrize("tol,bound", [(1e-10, 1e-8), (1e-13, 1e-11)])
def test_cn_fp32_refined(torch_cuda, tol, bound):
    """Precision form of CN: FP32 inner GMRES (operator, Krylov vectors, Jacobi) inside an FP64
    residual/refinement loop reaches the FP64 tolerance; trajectory vs the oracle's LU CN."""
    prob = W.shock(nx=15, npc=7, lmax=3)
    orc = NodalOracle(prob)
    sol = _solver(prob, "fp32")
    y = sol.initial_state()
    st = sol.step_cn(y, 1.0, 12, tol=tol, restart=30, maxit=4000)
    torch_cuda.cuda.synchronize()
    want = orc.cn(np.zeros(sol.N), 1.0, 12)
    err = np.linalg.norm(y.cpu().numpy() - want) / np.linalg.norm(want)
    assert st.last_rel_residual <= tol and err < bound, (err, st.last_rel_residual)


# ------------------------------------------------------------------------------------------------
# orders at the ends of the supported ranges, and degenerate systems
# ------------------------------------------------------------------------------------------------
_EDGE_ORDERS = {
    "k0_periodic1d": lambda: W.periodic_1d(ncells=5, k=0, lmax=2),
    "l0_periodic1d": lambda: W.periodic_1d(ncells=4, k=2, lmax=0),
    "l0_shock": lambda: W.shock(nx=4, npc=3, k=1, lmax=0, xr=(-2.0, 2.0), lnpr=(0.0, 2.0)),
    "l0_box_zero_operator": lambda: W.box3d(ncells=2, k=2, lmax=0),
    "k0_box": lambda: W.box3d(ncells=3, k=0, lmax=2),
    "l11_periodic1d": lambda: W.periodic_1d(ncells=2, k=1, lmax=11),
    "k4_shock": lambda: W.shock(nx=2, npc=2, k=4, lmax=1, xr=(-2.0, 2.0), lnpr=(0.0, 2.0)),
}


@pytest.mark.parametrize("name", list(_EDGE_ORDERS))
def test_apply_edge_orders(torch_cuda, name):
    """k = 0 and 4, l_max = 0 and 11 (l_max = 0 with U = 0 gives D = 0): every column of M^-1 D and
    of its transpose equals the oracle's, and the right-side mode M^-1 (h - D x) agrees."""
    from paper_2501_05110_gb300 import sapgpu
    torch = torch_cuda
    prob = _EDGE_ORDERS[name]()
    orc = NodalOracle(prob)
    sol = _solver(prob)
    N = sol.N
    assert N == orc.disc.N
    eye = np.eye(N)
    O = np.stack([orc.apply(eye[:, j]) for j in range(N)], axis=1)
    G = np.stack([_gpu_apply(torch, sol, eye[:, j]) for j in range(N)], axis=1)
    GT = []
    for j in range(N):
        x = torch.from_numpy(eye[:, j]).cuda()
        y = torch.empty_like(x)
        sol.apply(x, y, sapgpu.APPLY_T)
        GT.append(y.cpu().numpy())
    GT = np.stack(GT, axis=1)
    if not O.any():
        assert not G.any() and not GT.any()
    else:
        assert _rel_max(G, O) < 1e-12
        assert _rel_max(GT, O.T) < 1e-12
    y = np.random.default_rng(4).standard_normal(N)
    want = orc.apply(y, True)
    got = _gpu_apply(torch, sol, y, True)
    assert (not want.any() and not got.any()) or _rel_max(got, want) < 1e-12


def test_cn_zero_right_side_stays_zero(torch_cuda):
    """No source and a zero state: b = 0, so each CN step returns exactly zero without iterating."""
    torch = torch_cuda
    prob = W.shock(nx=15, npc=7, lmax=3, Q=0.0)
    sol = _solver(prob)
    y = torch.zeros(sol.N, dtype=torch.float64, device="cuda")
    st = sol.step_cn(y, 1.0, 3, 1e-10, 30, 100)
    torch.cuda.synchronize()
    assert not y.any()
    assert st.iterations == 0


# ------------------------------------------------------------------------------------------------
# transposed operator (discrete adjoint)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("idx", range(5))
def test_apply_transpose_tiny_vs_oracle(torch_cuda, idx):
    """Every column of (M^-1 D)^T from the library equals the transposed oracle operator."""
    from paper_2501_05110_gb300 import sapgpu
    prob = _tiny_problems()[idx]
    orc = NodalOracle(prob)
    sol = _solver(prob)
    N = sol.N
    eye = np.eye(N)
    O = np.stack([orc.apply(eye[:, j]) for j in range(N)], axis=1)
    GT = []
    for j in range(N):
        x = torch_cuda.from_numpy(eye[:, j]).cuda()
        y = torch_cuda.empty_like(x)
        sol.apply(x, y, sapgpu.APPLY_T)
        GT.append(y.cpu().numpy())
    GT = np.stack(GT, axis=1)
    assert _rel_max(GT, O.T) < 1e-12


@pytest.mark.parametrize("name", ["periodic1d", "shock_small", "box_small", "shock_graded"])
def test_apply_transpose_dot_product(torch_cuda, name):
    """<L x, y> = <x, L^T y> for random x, y."""
    from paper_2501_05110_gb300 import sapgpu
    torch = torch_cuda
    if name == "periodic1d":
        prob = W.periodic_1d()
    elif name == "shock_small":
        prob = W.shock(nx=15, npc=7, lmax=3)
    elif name == "box_small":
        prob = W.box3d(ncells=3, k=2, lmax=3)
    else:
        xe = np.concatenate([-np.geomspace(30, 0.05, 9), np.linspace(-0.04, 0.04, 5), np.geomspace(0.05, 60, 10)])
        prob = W.shock(x_edges=np.sort(xe), npc=6, lmax=2, lnpr=(-1.0, 4.0), Ls=0.05)
    sol = _solver(prob)
    g = torch.Generator(device="cuda").manual_seed(21)
    x = torch.randn(sol.N, device="cuda", dtype=torch.float64, generator=g)
    y = torch.randn(sol.N, device="cuda", dtype=torch.float64, generator=g)
    Lx, LTy = torch.empty_like(x), torch.empty_like(y)
    sol.apply(x, Lx, sapgpu.APPLY_D)
    sol.apply(y, LTy, sapgpu.APPLY_T)
    torch.cuda.synchronize()
    a, b = float(Lx @ y), float(x @ LTy)
    scale = float(Lx.abs() @ y.abs())
    assert abs(a - b) < 1e-13 * scale, (a, b)
