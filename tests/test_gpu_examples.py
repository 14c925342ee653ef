"""The paper's examples with known solutions that exercise truncation in l_max, run by the library.

* Advection in a constant magnetic field (Sec. 4.2): without scattering the particles gyrate, so
  the distribution returns to its initial state after every gyro-period T_g = 2 pi gamma / B0 in a
  static plasma, and after N periods in a periodic box of side L = N U0 T_g in a moving one.  The
  difference from the discrete initial state is the truncation error of the expansion; it must
  fall when l_max grows (3 -> 5).  A small mesh is checked against the oracle first (the 2-D,
  k = 3 shape runs the cell-node kernel).
* Closure (Sec. 4.3): free streaming of an isotropic Gaussian along x; the exact angular
  distribution at x = 6 sigma, t = 12/sqrt(3) follows from the characteristics,
  f = exp(-(x - V cos(theta) t)^2 / (2 sigma^2)) / (sqrt(2 pi) sigma).  The reconstruction
  sum_l f_l00 Y_l0(theta) from the library's coefficients converges to it as l_max grows (l_max = 11
  reproduces it); with scattering nu = 0.1 a lower l_max is closer to l_max = 11 than without.
"""
import math

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


def _run(torch, prob, nsteps):
    from paper_2501_05110_gb300 import sapgpu
    sol = sapgpu.Solver(prob)
    y0 = sol.initial_state()
    y = y0.clone()
    sol.step_erk(y, prob.dt, nsteps)
    torch.cuda.synchronize()
    return sol, y0.cpu().numpy(), y.cpu().numpy()


# ------------------------------------------------------------------------------------------------
# gyro-advection
# ------------------------------------------------------------------------------------------------
def test_gyro_small_vs_oracle(torch_cuda):
    prob = W.gyro_advection(ncells=6, k=3, lmax=3, dt=0.02)
    sol, y0, y = _run(torch_cuda, prob, 10)
    want = NodalOracle(prob).rk4(y0, prob.dt, 10)
    assert np.linalg.norm(y - want) < 1e-12 * np.linalg.norm(want)


def _residual_000(prob, y0, y):
    n, nloc = prob.n, (prob.k + 1) ** 2
    a = y.reshape(-1, n, nloc)[:, 0, :]
    b = y0.reshape(-1, n, nloc)[:, 0, :]
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_gyro_static_returns_after_gyro_periods(torch_cuda):
    """U0 = 0, 10 gyro-periods (t = 20): the residual against the discrete initial state is the
    truncation error, smaller for l_max = 5 than for l_max = 3."""
    res = {}
    for lmax in (3, 5):
        prob = W.gyro_advection(ncells=64, k=3, lmax=lmax, U0=0.0)
        _, y0, y = _run(torch_cuda, prob, 1000)
        res[lmax] = _residual_000(prob, y0, y)
    print(f"gyro static, t = 20: relative residual of f_000 {res}")
    # measured: 4.6e-6 (l_max = 3), 1.3e-6 (l_max = 5)
    assert res[5] < 0.5 * res[3], res
    assert res[3] < 3e-5, res


def test_gyro_moving_returns_after_100_periods(torch_cuda):
    """U0 = 0.1 in the box L = 20 = 100 U0 T_g: back at the start after t = 200 (10,000 steps), up to
    the truncation error at l_max = 3; particle number conserved."""
    prob = W.gyro_advection(ncells=64, k=3, lmax=3, U0=0.1)
    _, y0, y = _run(torch_cuda, prob, 10000)
    r = _residual_000(prob, y0, y)
    w = np.outer(*(2 * [np.polynomial.legendre.leggauss(4)[1] / 2])).ravel()
    mass = lambda v: float((v.reshape(-1, prob.n, 16)[:, 0, :] * w).sum())
    print(f"gyro moving, t = 200: relative residual of f_000 {r:.4e}; mass drift {abs(mass(y) - mass(y0)) / mass(y0):.3e}")
    assert r < 2e-4, r  # measured 3.0e-5
    assert abs(mass(y) - mass(y0)) < 1e-10 * abs(mass(y0))


# ------------------------------------------------------------------------------------------------
# closure
# ------------------------------------------------------------------------------------------------
def _angular_at(prob, y, x0, thetas):
    """f_h(x0, theta) = sum_l f_l00(x0) Y_l0(theta): the Lagrange interpolant through the cell's
    Gauss nodes at x0, then the (axisymmetric) spherical-harmonic sum."""
    from oracle import sh
    e = prob.edges[0]
    c = int(np.searchsorted(e, x0, side="right") - 1)
    q = prob.k + 1
    xg = 0.5 * (np.polynomial.legendre.leggauss(q)[0] + 1.0)
    t = (x0 - e[c]) / (e[c + 1] - e[c])
    lag = np.array([np.prod([(t - xg[j]) / (xg[i] - xg[j]) for j in range(q) if j != i]) for i in range(q)])
    coef = y.reshape(-1, prob.n, q)[c] @ lag  # value of every coefficient at x0
    f = np.zeros_like(thetas)
    for l in range(prob.lmax + 1):
        f += coef[sh.index_map(l, 0, 0)] * sh.real_Y(l, 0, 0, thetas, 0.0)
    return f


def _exact(x, t, thetas, sigma=1.0, V=math.sqrt(3.0) / 2):
    return np.exp(-(x - V * np.cos(thetas) * t) ** 2 / (2 * sigma ** 2)) / (math.sqrt(2 * math.pi) * sigma)


def test_closure_converges_to_characteristics(torch_cuda):
    thetas = np.linspace(0.0, math.pi, 151)
    tF = 12.0 / math.sqrt(3.0)
    want = _exact(6.0, tF, thetas)
    errs = {}
    for lmax in (3, 7, 11):
        prob = W.closure(lmax=lmax)
        _, _, y = _run(torch_cuda, prob, prob.nsteps)
        errs[lmax] = float(np.abs(_angular_at(prob, y, 6.0, thetas) - want).max() / want.max())
    print(f"closure, x = 6, t = 12/sqrt(3): max relative error of f(theta) {errs}")
    # measured: 0.19 (l_max = 3), 0.078 (7), 0.017 (11)
    assert errs[11] < errs[7] < errs[3], errs
    assert errs[11] < 0.04, errs


def test_closure_scattering_needs_lower_lmax(torch_cuda):
    """With nu = 0.1 the l_max = 7 reconstruction is closer to l_max = 11 than without scattering."""
    thetas = np.linspace(0.0, math.pi, 151)
    gap = {}
    for nu in (0.0, 0.1):
        fs = {}
        for lmax in (7, 11):
            prob = W.closure(lmax=lmax, nu=nu)
            _, _, y = _run(torch_cuda, prob, prob.nsteps)
            fs[lmax] = _angular_at(prob, y, 6.0, thetas)
        gap[nu] = float(np.abs(fs[7] - fs[11]).max() / np.abs(fs[11]).max())
    print(f"closure, |f(l_max=7) - f(l_max=11)| / max f: {gap}")
    assert gap[0.1] < 0.1 * gap[0.0], gap  # measured 1.8e-4 against 0.096
