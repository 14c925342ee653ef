"""Boundary entry points: fields from device arrays on a stream (sap_set_fields_device) give the
same operator as fields from host arrays, and the theta-method at theta = 1/2 is sap_step_cn."""
import numpy as np
import pytest

from paper_2501_05110_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2501_05110_gb300 import build as sap_build
    sap_build.build()
    return torch


@pytest.mark.parametrize("name", ["shock", "box"])
def test_set_fields_device_equals_host(torch_cuda, name):
    from paper_2501_05110_gb300 import sapgpu
    torch = torch_cuda
    prob = W.shock(nx=15, npc=7, lmax=3) if name == "shock" else W.box3d(ncells=3, k=2, lmax=3)
    host = sapgpu.Solver(prob)
    dev = sapgpu.Solver(prob)
    f = dev.field_arrays(prob)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        # the field tensors are produced on `stream`; the call reads them after that work
        tensors = {k: (None if v is None else torch.from_numpy(v).to("cuda", non_blocking=False) * 1.0)
                   for k, v in f.items()}
        dev.set_fields_device(tensors, stream=stream)
    x = torch.from_numpy(np.random.default_rng(3).standard_normal(host.N)).cuda()
    a, b = torch.empty_like(x), torch.empty_like(x)
    for mode in (sapgpu.APPLY_D, sapgpu.APPLY_RHS, sapgpu.APPLY_T):
        host.apply(x, a, mode)
        dev.apply(x, b, mode)
        torch.cuda.synchronize()
        assert torch.equal(a, b), mode


def test_theta_half_is_crank_nicolson(torch_cuda):
    from paper_2501_05110_gb300 import sapgpu
    torch = torch_cuda
    prob = W.shock(nx=15, npc=7, lmax=3)
    s1, s2 = sapgpu.Solver(prob), sapgpu.Solver(prob)
    y1, y2 = s1.initial_state(), s2.initial_state()
    st1 = s1.step_cn(y1, 1.0, 4, tol=1e-12)
    st2 = s2.step_theta(y2, 1.0, 0.5, 4, tol=1e-12)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2) and st1.iterations == st2.iterations


def test_theta_rejects_bad_values(torch_cuda):
    from paper_2501_05110_gb300 import sapgpu
    torch = torch_cuda
    prob = W.shock(nx=5, npc=3, lmax=1)
    sol = sapgpu.Solver(prob)
    y = sol.initial_state()
    for th in (-0.1, 1.5, float("nan")):
        with pytest.raises(sapgpu.SapError) as e:
            sol.step_theta(y, 1.0, th, 1)
        assert e.value.status == sapgpu.SAP_EINVAL
    batch = sapgpu.Batch([prob, W.shock(nx=4, npc=3, lmax=2)], "fp64")
    yb = batch.initial_state()
    with pytest.raises(sapgpu.SapError) as e:
        batch.step_theta(yb, 1.0, 1.0, 1)
    assert e.value.status == sapgpu.SAP_EUNSUPPORTED
    torch.cuda.synchronize()
