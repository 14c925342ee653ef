"""Batched runs (sap_create_batch): independent shock instances with different lmax, meshes,
compression ratios and scattering rates, run by one launch per operator apply and lock-step
per-instance GMRES.  Checked against single-instance runs and against the oracle per instance."""
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


def _instances():
    return [
        W.shock(nx=7, npc=4, lmax=1, r=2.5, nu0=0.3, name="b0"),
        W.shock(nx=9, npc=5, lmax=3, r=4.0, nu0=2.0, name="b1"),
        W.shock(nx=6, npc=4, lmax=2, r=3.0, nu0=1.0, name="b2"),
        W.shock(nx=5, npc=3, lmax=5, r=3.5, nu0=0.5, name="b3"),
    ]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_apply_equals_single(torch_cuda, prec):
    from paper_2501_05110_gb300 import sapgpu
    torch = torch_cuda
    probs = _instances()
    batch = sapgpu.Batch(probs, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    g = torch.Generator(device="cuda").manual_seed(9)
    x = torch.randn(batch.N, device="cuda", dtype=torch.float64, generator=g).to(dt)
    y = torch.empty_like(x)
    batch.apply(x, y)
    torch.cuda.synchronize()
    for p, xi, yi in zip(probs, batch.split(x), batch.split(y)):
        s = sapgpu.Solver(p, prec)
        ys = torch.empty_like(xi)
        s.apply(xi.contiguous(), ys)
        torch.cuda.synchronize()
        assert torch.equal(ys, yi), p.name


def test_batched_cn_fp64_matches_oracle(torch_cuda):
    from paper_2501_05110_gb300 import sapgpu
    probs = _instances()
    batch = sapgpu.Batch(probs, "fp64")
    y = batch.initial_state()
    st = batch.step_cn(y, 1.0, 8, tol=1e-13, restart=30, maxit=4000)
    torch_cuda.cuda.synchronize()
    assert st.last_rel_residual <= 1e-13
    for p, yi in zip(probs, batch.split(y)):
        want = NodalOracle(p).cn(np.zeros(yi.numel()), 1.0, 8)
        err = np.linalg.norm(yi.cpu().numpy() - want) / np.linalg.norm(want)
        assert err < 1e-11, (p.name, err)


def test_batched_cn_fp32_refined_matches_oracle(torch_cuda):
    from paper_2501_05110_gb300 import sapgpu
    probs = _instances()
    batch = sapgpu.Batch(probs, "fp32")
    y = batch.initial_state()
    st = batch.step_cn(y, 1.0, 8, tol=1e-10, restart=30, maxit=4000)
    torch_cuda.cuda.synchronize()
    assert st.last_rel_residual <= 1e-10
    for p, yi in zip(probs, batch.split(y)):
        want = NodalOracle(p).cn(np.zeros(yi.numel()), 1.0, 8)
        err = np.linalg.norm(yi.cpu().numpy() - want) / np.linalg.norm(want)
        assert err < 1e-8, (p.name, err)


def test_batched_erk_equals_single(torch_cuda):
    from paper_2501_05110_gb300 import sapgpu
    torch = torch_cuda
    probs = _instances()
    batch = sapgpu.Batch(probs, "fp64")
    g = torch.Generator(device="cuda").manual_seed(4)
    y = torch.randn(batch.N, device="cuda", dtype=torch.float64, generator=g)
    ys = [yi.clone() for yi in batch.split(y)]
    batch.step_erk(y, 0.01, 3)
    torch.cuda.synchronize()
    for p, yi, y0 in zip(probs, batch.split(y), ys):
        s = sapgpu.Solver(p, "fp64")
        s.step_erk(y0, 0.01, 3)
        torch.cuda.synchronize()
        assert torch.equal(y0, yi), p.name
