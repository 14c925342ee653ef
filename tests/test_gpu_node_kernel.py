"""The node kernel (uniform.cu): the operator apply for spatial 3-D problems with k = 2 whose term
coefficients are all uniform, run with the combined coupling matrices R, beta_a, |beta_a| as compiled
sparse patterns.  It must give the oracle's operator (Eq. definition-mass-and-dg-matrix with the
upwind flux, Eq. definition-upwind-flux) like the row kernel does:

* which kernel runs: the box runs the node kernel, the shock and k != 2 boxes the row kernel, and
  sap_set_apply_kernel("rows") switches it off;
* y = M^-1 D x and y = M^-1 (h - D x) for l_max = 1..5 on 3^3 (and 4 x 3 x 5, graded) boxes with
  periodic, zero-inflow and continuous boundaries, uniform U along an oblique direction (|beta| of
  W |U + lam V| W^T) and a source, FP64 to 1e-12 and FP32 to 1e-5 of the largest output;
* the same states through both kernels agree to FP64 rounding; RK4 steps through the node kernel equal
  the oracle's RK4; the FP32 precision form and a CN step run through it.
"""
import dataclasses

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


def _box(lmax, case="periodic"):
    prob = W.box3d(ncells=3, k=2, lmax=lmax)
    if case == "periodic":
        return prob
    if case == "mixed_bc":
        return dataclasses.replace(prob, bc=[("inflow0", "continuous"), ("continuous", "inflow0"), ("periodic", "periodic")])
    if case == "graded_src_U":
        # 4 x 3 x 5 cells, graded in x, uniform U along (0.3, -0.2, 0.1), a uniform source
        ex = np.array([-10.0, -7.0, -1.0, 2.0, 10.0])
        ey = np.linspace(-10.0, 10.0, 4)
        ez = np.linspace(-10.0, 10.0, 6)
        return dataclasses.replace(prob, edges=[ex, ey, ez], U=W._const3([0.3, -0.2, 0.1]), s000=W._scalar(0.25),
                                   terms=frozenset({"adv", "rot", "coll", "src"}),
                                   bc=[("inflow0", "inflow0"), ("periodic", "periodic"), ("continuous", "continuous")])
    raise ValueError(case)


def _apply(torch, sol, y, mode, dtype):
    x = torch.from_numpy(y).to("cuda", dtype)
    out = torch.empty_like(x)
    sol.apply(x, out, mode)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


def _rel_max(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_kernel_in_use(torch_cuda):
    from paper_2501_05110_gb300 import sapgpu
    box = sapgpu.Solver(_box(3))
    assert box.apply_kernel_in_use() == "node"
    box.set_apply_kernel("rows")
    assert box.apply_kernel_in_use() == "rows"
    box.set_apply_kernel("auto", 2)
    assert box.apply_kernel_in_use() == "node"
    assert sapgpu.Solver(W.shock(nx=5, npc=3, lmax=1)).apply_kernel_in_use() == "rows"
    assert sapgpu.Solver(W.box3d(ncells=2, k=1, lmax=2)).apply_kernel_in_use() == "rows"
    assert sapgpu.Solver(W.box3d(ncells=2, k=2, lmax=0)).apply_kernel_in_use() == "rows"


@pytest.mark.parametrize("lmax", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("case", ["periodic", "mixed_bc", "graded_src_U"])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_node_apply_vs_oracle(torch_cuda, lmax, case, prec, tol):
    from paper_2501_05110_gb300 import sapgpu
    torch = torch_cuda
    prob = _box(lmax, case)
    sol = sapgpu.Solver(prob, prec)
    kernel = sol.apply_kernel_in_use()
    if case != "graded_src_U":
        assert kernel == "node"
    orc = NodalOracle(prob)
    y = np.random.default_rng(100 + lmax).standard_normal(sol.N)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    for mode, rhs in ((sapgpu.APPLY_D, False), (sapgpu.APPLY_RHS, True)):
        got = _apply(torch, sol, y, mode, dtype)
        want = orc.apply(y, rhs=rhs)
        err = _rel_max(got, want)
        assert err < tol, (kernel, mode, err)
    sol.close()


@pytest.mark.parametrize("lmax", [3, 5])
@pytest.mark.parametrize("cells", [1, 3, 0])
def test_node_equals_rows(torch_cuda, lmax, cells):
    """The same state through both kernels (and through ragged last blocks: 27 cells with 1, 3 or the
    default cells per block): equal to FP64 rounding."""
    from paper_2501_05110_gb300 import sapgpu
    torch = torch_cuda
    prob = _box(lmax, "mixed_bc")
    sol = sapgpu.Solver(prob)
    y = np.random.default_rng(7).standard_normal(sol.N)
    sol.set_apply_kernel("auto", cells)
    a = _apply(torch, sol, y, sapgpu.APPLY_D, torch.float64)
    sol.set_apply_kernel("rows")
    b = _apply(torch, sol, y, sapgpu.APPLY_D, torch.float64)
    assert _rel_max(a, b) < 1e-13


def test_node_rk4_vs_oracle(torch_cuda):
    from paper_2501_05110_gb300 import sapgpu
    torch = torch_cuda
    prob = _box(3, "graded_src_U")
    prob = dataclasses.replace(prob, U=W._const3([0.0, 0.0, 0.0]))  # U = 0: the node kernel
    sol = sapgpu.Solver(prob)
    assert sol.apply_kernel_in_use() == "node"
    y0 = sol.initial_state()
    y = y0.clone()
    sol.step_erk(y, 0.01, 10)
    torch.cuda.synchronize()
    want = NodalOracle(prob).rk4(y0.cpu().numpy(), 0.01, 10)
    err = np.linalg.norm(y.cpu().numpy() - want) / np.linalg.norm(want)
    assert err < 1e-12, err


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-8)])
def test_node_cn_vs_oracle(torch_cuda, prec, tol):
    """CN steps (GMRES with the point-Jacobi diagonal from the combined reaction matrix) through the
    node kernel against the oracle's exact CN solve; the FP32 form refines in FP64."""
    from paper_2501_05110_gb300 import sapgpu
    torch = torch_cuda
    prob = _box(2, "mixed_bc")
    sol = sapgpu.Solver(prob, prec)
    assert sol.apply_kernel_in_use() == "node"
    y0 = sol.initial_state()
    y = y0.clone()
    sol.step_cn(y, 0.5, 3, tol=1e-13, restart=30, maxit=2000)
    torch.cuda.synchronize()
    want = NodalOracle(prob).cn(y0.cpu().numpy(), 0.5, 3)
    err = np.linalg.norm(y.cpu().numpy() - want) / np.linalg.norm(want)
    assert err < tol, err
