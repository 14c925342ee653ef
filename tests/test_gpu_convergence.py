"""The convergence study of Sec. 4.1 run by the library: the l_max = 1 system with B along z in a
periodic box, whose truncated-PDE solution is known in closed form (tests/test_oracle_pins.py
``_convergence_problem``).

* space: RK4 (sap_step_erk) with k = 1..5; the error of f_000 against the closed form falls as
  Delta x^(k+1) (least-squares slope over the meshes), and every run equals the oracle's RK4 run
  on the same mesh to 1e-12;
* time: the theta-method (sap_step_theta) with theta = 0, 1/2, 1 at k = 4; the largest error over the
  steps falls with orders 1, 2, 1, and the trajectory equals the oracle's theta-method (sparse LU)."""
import math

import numpy as np
import pytest

from .oracle_bridge import NodalOracle
from .test_oracle_pins import CONV_FINEST, CONV_SPACE, _convergence_problem, convergence_order

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2501_05110_gb300 import build as sap_build
    sap_build.build()
    return torch


def _err000(y, ex, t, k, nc, sol, Lbox=20.0):
    """Relative L2 error of f_000 at the Gauss points (the library's nodes)."""
    from paper_2501_05110_gb300 import sapgpu
    f = y.reshape(nc, 4, k + 1)[:, 0, :]
    x = sol.points(sapgpu.PTS_PHASE)[:, 0].reshape(nc, k + 1)
    w = np.polynomial.legendre.leggauss(k + 1)[1] / 2 * (Lbox / nc)
    return math.sqrt(np.sum(w * (f - ex(t, x)) ** 2)) / math.sqrt(np.sum(w * f ** 2))


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_gpu_convergence_space(torch_cuda, k):
    from paper_2501_05110_gb300 import sapgpu
    ncs, dt = CONV_SPACE[k]
    nsteps = int(round(1.0 / dt))
    errs = []
    for nc in ncs:
        prob, ex = _convergence_problem(nc, k)
        sol = sapgpu.Solver(prob)
        y0 = sol.initial_state()
        y = y0.clone()
        sol.step_erk(y, dt, nsteps)
        torch_cuda.cuda.synchronize()
        got = y.cpu().numpy()
        errs.append(_err000(got, ex, 1.0, k, nc, sol))
        if nc == 8:
            want = NodalOracle(prob).rk4(y0.cpu().numpy(), dt, nsteps)
            assert np.linalg.norm(got - want) < 1e-12 * np.linalg.norm(want)
        sol.close()
    print(f"space k={k}: errors {errs}, order {convergence_order(ncs, errs):.2f}")
    assert convergence_order(ncs, errs) > k + 1 - 0.3, errs
    assert errs[-1] < CONV_FINEST[k], errs


@pytest.mark.parametrize("theta,order", [(0.5, 2), (1.0, 1), (0.0, 1)])
def test_gpu_convergence_time(torch_cuda, theta, order):
    from paper_2501_05110_gb300 import sapgpu
    k, nc, tF = 4, 16, 2.0
    prob, ex = _convergence_problem(nc, k)
    orc = NodalOracle(prob)
    dts = (0.004, 0.002, 0.001) if theta == 0.0 else (0.04, 0.02, 0.01)
    errs = []
    for dt in dts:
        sol = sapgpu.Solver(prob)
        y = sol.initial_state()
        y0 = y.cpu().numpy()
        worst = 0.0
        nsteps = int(round(tF / dt))
        for i in range(1, nsteps + 1):
            sol.step_theta(y, dt, theta, 1, tol=1e-13, restart=30, maxit=4000)
            worst = max(worst, _err000(y.cpu().numpy(), ex, i * dt, k, nc, sol))
        errs.append(worst)
        if dt == dts[0]:
            d = orc.disc
            from oracle import steppers
            z = steppers.theta_method(d.M, d.D, d.h, d.from_gauss_nodal(y0), dt, nsteps, theta=theta)
            want = d.to_gauss_nodal(z)
            assert np.linalg.norm(y.cpu().numpy() - want) < 1e-11 * np.linalg.norm(want)
        sol.close()
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    print(f"time theta={theta}: errors {errs}, orders {orders}")
    assert all(abs(o - order) < 0.25 for o in orders), (errs, orders)
