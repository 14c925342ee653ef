"""Host logic of the trajectory adjoints (checkpoint segments, recomputation, the pairing of states
with steps, the accumulation of field gradients and the final chain rule to U1) on the CPU:
CNTrajectory and ERKTrajectory drive a small dense stand-in for the library solver, and their
gradients must equal torch autograd through the same dense trajectory, for every checkpoint
interval."""
import numpy as np
import pytest
import torch

from paper_2501_05110_gb300 import adjoint

N, NPV, NSTEPS = 12, 4, 7


class _Stats:
    iterations = 0


class _Model:
    """L(nu, U1) = L0 + diag(c * nu[node]) + U1 B, source s, initial state y0 (seeded)."""

    def __init__(self):
        rng = np.random.default_rng(0)
        self.L0 = torch.from_numpy(0.3 * rng.standard_normal((N, N)) + 2.0 * np.eye(N))
        self.B = torch.from_numpy(0.2 * rng.standard_normal((N, N)))
        self.c = torch.from_numpy(rng.uniform(0.5, 1.5, N))
        self.node = torch.from_numpy(np.arange(N) % NPV)
        self.s = torch.from_numpy(rng.standard_normal(N))
        self.y0 = torch.from_numpy(rng.standard_normal(N))

    def L(self, nu, u1):
        nu = torch.as_tensor(nu, dtype=torch.float64)
        return self.L0 + torch.diag(self.c * nu[self.node]) + u1 * self.B


class _FakeSolver:
    """Dense stand-in for sapgpu.Solver with the library's step and adjoint-step semantics.  Its one
    spatial "field" U (a single value) enters L as U B; its derivative problem has dU/dU1 = 2 U1
    (the model is evaluated at U = U1^2), which exercises the chain rule's use of the field
    derivative."""

    def __init__(self, model, nu, u1):
        self.m, self.A = model, model.L(nu, u1 ** 2)
        self.u1 = u1

    def initial_state(self):
        return self.m.y0.clone()

    def apply(self, x, out, mode=0):
        out.copy_(self.A @ x)

    def _F(self, y):
        return self.m.s - self.A @ y

    def step_erk(self, y, dt, nsteps):
        for _ in range(nsteps):
            k1 = self._F(y)
            k2 = self._F(y + 0.5 * dt * k1)
            k3 = self._F(y + 0.5 * dt * k2)
            k4 = self._F(y + dt * k3)
            y.copy_(y + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4))

    def step_cn(self, y, dt, nsteps, tol, restart, maxit):
        I = torch.eye(N, dtype=torch.float64)
        for _ in range(nsteps):
            y.copy_(torch.linalg.solve(I + 0.5 * dt * self.A, (I - 0.5 * dt * self.A) @ y + dt * self.m.s))
        return _Stats()

    def _grad_add(self, grad_nu, coef, a, z):
        grad_nu.index_add_(0, self.m.node, coef * self.m.c * a * z)

    def adjoint_step_cn(self, zp, zn, lam, dt, tol, restart, maxit, mu_out=None, grad_nu=None):
        I = torch.eye(N, dtype=torch.float64)
        mu = torch.linalg.solve((I + 0.5 * dt * self.A).T, lam)
        lam.copy_((I - 0.5 * dt * self.A).T @ mu)
        if mu_out is not None:
            mu_out.copy_(mu)
        if grad_nu is not None:
            self._grad_add(grad_nu, -0.5 * dt, mu, zp + zn)
        return _Stats()

    def adjoint_step_erk(self, y, lam, dt, grad_nu=None, stages_out=None):
        AT = self.A.T
        Y2 = y + 0.5 * dt * self._F(y)
        Y3 = y + 0.5 * dt * self._F(Y2)
        Y4 = y + dt * self._F(Y3)
        kb4 = dt / 6 * lam
        kb3 = dt / 3 * lam - dt * (AT @ kb4)
        kb2 = dt / 3 * lam - 0.5 * dt * (AT @ kb3)
        kb1 = dt / 6 * lam - 0.5 * dt * (AT @ kb2)
        if grad_nu is not None:
            for kb, Y in ((kb1, y), (kb2, Y2), (kb3, Y3), (kb4, Y4)):
                self._grad_add(grad_nu, -1.0, kb, Y)
        if stages_out is not None:
            stages_out.copy_(torch.cat([Y2, Y3, Y4, kb1, kb2, kb3, kb4]))
        lam.copy_(lam - AT @ (kb1 + kb2 + kb3 + kb4))
        return _Stats()

    def field_grad_buffers(self, device="cpu", which=()):
        out = {k: None for k in which}
        out["U"] = torch.zeros(1, dtype=torch.float64)
        out["nu"] = torch.zeros(NPV, dtype=torch.float64)
        return out

    def field_arrays(self, prob):
        return {"U": np.array([prob])}  # the fake derivative problem is the number dU/dU1

    def adjoint_step(self, scheme, zp, zn, lam, dt, grads, tol=1e-12, restart=30, maxit=4000):
        B = self.m.B
        if scheme == "cn":
            I = torch.eye(N, dtype=torch.float64)
            mu = torch.linalg.solve((I + 0.5 * dt * self.A).T, lam)
            lam.copy_((I - 0.5 * dt * self.A).T @ mu)
            self._grad_add(grads["nu"], -0.5 * dt, mu, zp + zn)
            grads["U"] += -0.5 * dt * (mu @ (B @ (zp + zn)))
        else:
            AT = self.A.T
            Y2 = zp + 0.5 * dt * self._F(zp)
            Y3 = zp + 0.5 * dt * self._F(Y2)
            Y4 = zp + dt * self._F(Y3)
            kb4 = dt / 6 * lam
            kb3 = dt / 3 * lam - dt * (AT @ kb4)
            kb2 = dt / 3 * lam - 0.5 * dt * (AT @ kb3)
            kb1 = dt / 6 * lam - 0.5 * dt * (AT @ kb2)
            for kb, Y in ((kb1, zp), (kb2, Y2), (kb3, Y3), (kb4, Y4)):
                self._grad_add(grads["nu"], -1.0, kb, Y)
                grads["U"] += -(kb @ (B @ Y))
            lam.copy_(lam - AT @ (kb1 + kb2 + kb3 + kb4))
        return _Stats()

    def close(self):
        pass


class _FakeFamily(adjoint.CNProblemFamily):
    def solver(self, nu_nodes, U1):
        return _FakeSolver(self.make_problem, nu_nodes, U1)

    def field_derivative(self, nu_nodes, U1):
        return 2.0 * U1  # dU/dU1 of the fake's field U = U1^2


def _reference(model, scheme, dt, w, nu0, u10):
    nu = torch.tensor(nu0, requires_grad=True)
    u1 = torch.tensor(u10, dtype=torch.float64, requires_grad=True)
    A = model.L0 + torch.diag(model.c * nu[model.node]) + u1 ** 2 * model.B
    I = torch.eye(N, dtype=torch.float64)
    F = lambda y: model.s - A @ y
    y = model.y0.clone()
    for _ in range(NSTEPS):
        if scheme == "erk":
            k1 = F(y); k2 = F(y + 0.5 * dt * k1); k3 = F(y + 0.5 * dt * k2); k4 = F(y + dt * k3)
            y = y + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        else:
            y = torch.linalg.solve(I + 0.5 * dt * A, (I - 0.5 * dt * A) @ y + dt * model.s)
    (w @ y).backward()
    return nu.grad.numpy(), float(u1.grad)


@pytest.mark.parametrize("scheme", ["erk", "cn"])
@pytest.mark.parametrize("checkpoint", [1, 2, 3, 50])
def test_trajectory_adjoint_matches_autograd(scheme, checkpoint):
    model = _Model()
    dt = 0.1 if scheme == "erk" else 0.5
    w = torch.from_numpy(np.random.default_rng(1).standard_normal(N))
    nu0 = np.random.default_rng(2).uniform(0.5, 2.0, NPV)
    fam = _FakeFamily(make_problem=model, nsteps=NSTEPS, dt=dt, checkpoint=checkpoint)
    nu_t = torch.tensor(nu0, requires_grad=True)
    u1_t = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
    fn = adjoint.ERKTrajectory if scheme == "erk" else adjoint.CNTrajectory
    (w @ fn.apply(nu_t, u1_t, fam)).backward()
    g_nu, g_u1 = _reference(model, scheme, dt, w, nu0, 0.3)
    np.testing.assert_allclose(nu_t.grad.numpy(), g_nu, rtol=1e-11, atol=1e-13 * np.abs(g_nu).max())
    assert abs(float(u1_t.grad) - g_u1) < 1e-11 * abs(g_u1)
