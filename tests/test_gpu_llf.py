"""The local Lax--Friedrichs flux (sap_set_flux(SAP_FLUX_LLF)) against the oracle: every column of
L = M^-1 D and of L^T on small meshes of each face route (constant |beta| matrix in 1-D and 3-D,
the eigen route on spatial faces and the per-point route on momentum faces of the shock), random
inputs on a graded shock, and exactly solved CN trajectories; the adjoint's field gradients are
refused for it."""
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


def _llf(prob):
    return dataclasses.replace(prob, flux="llf")


_CASES = {
    "periodic1d": lambda: W.periodic_1d(ncells=3, k=2, lmax=2),
    "shock_lnp": lambda: W.shock(nx=3, npc=3, lmax=2, xr=(-2.0, 2.0), lnpr=(0.0, 2.0)),
    "shock_p": lambda: W.shock(nx=3, npc=2, lmax=1, xr=(-2.0, 2.0), lnpr=(0.0, 2.0), momentum="p"),
    "box": lambda: W.box3d(ncells=2, k=1, lmax=1),
}


@pytest.mark.parametrize("name", list(_CASES))
def test_llf_columns_vs_oracle(torch_cuda, name):
    from paper_2501_05110_gb300 import sapgpu
    torch = torch_cuda
    prob = _llf(_CASES[name]())
    orc = NodalOracle(prob)
    sol = sapgpu.Solver(prob)
    N = sol.N
    eye = np.eye(N)
    O = np.stack([orc.apply(eye[:, j]) for j in range(N)], axis=1)
    G, GT = [], []
    for j in range(N):
        x = torch.from_numpy(eye[:, j]).cuda()
        y = torch.empty_like(x)
        sol.apply(x, y, sapgpu.APPLY_D)
        G.append(y.cpu().numpy())
        sol.apply(x, y, sapgpu.APPLY_T)
        GT.append(y.cpu().numpy())
    G, GT = np.stack(G, axis=1), np.stack(GT, axis=1)
    scale = np.abs(O).max()
    assert np.abs(G - O).max() < 1e-12 * scale
    assert np.abs(GT - O.T).max() < 1e-12 * scale
    # the flux matters here: the upwind operator differs
    Ou = np.stack([NodalOracle(_CASES[name]()).apply(eye[:, j]) for j in range(N)], axis=1)
    assert np.abs(Ou - O).max() > 1e-6 * scale


@pytest.mark.parametrize("prec,bound", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_llf_random_graded_shock(torch_cuda, prec, bound):
    from paper_2501_05110_gb300 import sapgpu
    torch = torch_cuda
    xe = np.concatenate([-np.geomspace(30, 0.05, 9), np.linspace(-0.04, 0.04, 5), np.geomspace(0.05, 60, 10)])
    prob = _llf(W.shock(x_edges=np.sort(xe), npc=6, lmax=2, lnpr=(-1.0, 4.0), Ls=0.05))
    sol = sapgpu.Solver(prob, prec)
    y = np.random.default_rng(13).standard_normal(sol.N)
    x = torch.from_numpy(y).to("cuda", torch.float64 if prec == "fp64" else torch.float32)
    out = torch.empty_like(x)
    for mode, rhs in ((sapgpu.APPLY_D, False), (sapgpu.APPLY_RHS, True)):
        sol.apply(x, out, mode)
        torch.cuda.synchronize()
        want = NodalOracle(prob).apply(y, rhs)
        assert np.abs(out.double().cpu().numpy() - want).max() < bound * np.abs(want).max()


def test_llf_cn_vs_oracle(torch_cuda):
    from paper_2501_05110_gb300 import sapgpu
    prob = _llf(W.shock(nx=15, npc=7, lmax=3))
    sol = sapgpu.Solver(prob)
    y = sol.initial_state()
    sol.step_cn(y, 1.0, 6, tol=1e-14, restart=30, maxit=4000)
    torch_cuda.cuda.synchronize()
    want = NodalOracle(prob).cn(np.zeros(sol.N), 1.0, 6)
    err = np.linalg.norm(y.cpu().numpy() - want) / np.linalg.norm(want)
    print(f"LLF CN vs oracle: {err:.3e}")
    assert err < 1e-12, err


def test_llf_adjoint_field_gradients_refused(torch_cuda):
    from paper_2501_05110_gb300 import sapgpu
    torch = torch_cuda
    prob = _llf(W.shock(nx=5, npc=3, lmax=1))
    sol = sapgpu.Solver(prob)
    y = sol.initial_state()
    lam = torch.ones(sol.N, dtype=torch.float64, device="cuda")
    grads = sol.field_grad_buffers()
    with pytest.raises(sapgpu.SapError) as e:
        sol.adjoint_step("cn", y, y, lam, 1.0, grads)
    assert e.value.status == sapgpu.SAP_EUNSUPPORTED
    # the nu gradient alone (linear in nu) is still formed
    g = {"nu": grads["nu"]}
    sol.adjoint_step("cn", y, y, lam, 1.0, g)
