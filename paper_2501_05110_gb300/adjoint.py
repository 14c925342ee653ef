"""Discrete adjoints of Crank--Nicolson and RK4 trajectories as torch.autograd.Functions.

The forward pass runs the steps in the library (sap_step_cn / sap_step_erk) and keeps the state
every `checkpoint` steps.  The backward pass walks the segments from the end: it recomputes a
segment's states from its checkpoint and runs the library's adjoint step (sap_adjoint_step) through
them.  Per CN step (theta = 1/2 of Eq. theta-method) the library solves A^T mu = lambda_n, sets
lambda_{n-1} = B^T mu and adds the exact gradients of J with respect to every prescribed field at its
sampling points, -dt/2 mu^T (dL/dfield)(zeta_{n-1} + zeta_n); per RK4 step (Sec. 3.4) it recomputes
the stage inputs, forms the stage adjoints kb_i and adds -sum_i kb_i^T (dL/dfield) Y_i.  The upwind
matrices are differentiated by the Daleckii--Krein formula inside the library.

The parameters reach the fields by the chain rule, done here once per backward pass:
  dJ/dnu   is the library's nodal nu-gradient itself (nu is given per phase-space node);
  dJ/dU1 = sum over the field arrays of <dJ/dfield, dfield/dU1>, with dfield/dU1 evaluated at the
           library's points from the problem family (for the shock: U, grad U linear in U1, (U.grad)U
           quadratic).
Only argument marshalling, the checkpoint bookkeeping and this final chain rule live here; every
operator apply, linear solve and gradient accumulation runs in libsapgpu.so.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable, Optional

import torch

from . import sapgpu
from . import workloads

# field arrays through which the shock speed enters (sap_field_grads members)
U1_FIELDS = ("U", "gradU", "DUDt", "Uface0", "Uface1", "Uface2")


@dataclasses.dataclass
class CNProblemFamily:
    """A problem parametrised by a per-node nu (library phase-node order) and the shock speed, with
    the time stepping of a trajectory (tol and restart apply to CN only)."""
    make_problem: Callable  # (nu_nodes_numpy or None, U1) -> workloads.Problem
    nsteps: int
    dt: float
    tol: float = 1e-12
    restart: int = 30
    checkpoint: int = 50
    # (nu_nodes_numpy or None, U1) -> Problem whose fields are d(field)/dU1 at any point; None: the
    # shock family's own (workloads.shock_U1_derivative)
    make_field_derivative: Optional[Callable] = None
    # filled by the backward pass: wall time of its parts (s) and the adjoint GMRES iterations per step
    last_backward: dict = dataclasses.field(default_factory=dict)

    def solver(self, nu_nodes, U1):
        return sapgpu.Solver(self.make_problem(nu_nodes, U1), "fp64")

    def field_derivative(self, nu_nodes, U1):
        if self.make_field_derivative is not None:
            return self.make_field_derivative(nu_nodes, U1)
        return workloads.shock_U1_derivative(self.make_problem(nu_nodes, U1), U1)


def _chain_u1(grads, dfields, device):
    """dJ/dU1 = sum_k <dJ/dfield_k, dfield_k/dU1> (one device reduction per field array)."""
    total = torch.zeros((), dtype=torch.float64, device=device)
    for k in U1_FIELDS:
        g, d = grads.get(k), dfields.get(k)
        if g is not None and d is not None:
            total = total + g @ torch.as_tensor(d, dtype=torch.float64, device=device)
    return total


class CNTrajectory(torch.autograd.Function):
    """zeta_N = CN^N(zeta_0 = initial state; nu, U1).  Inputs: nu_nodes (npv, float64, cuda),
    U1 (0-d float64 tensor).  Returns the final state (N, float64, cuda)."""

    @staticmethod
    def forward(ctx, nu_nodes, U1, fam: CNProblemFamily):
        u1 = float(U1)
        nu_np = nu_nodes.detach().cpu().numpy()
        sol = fam.solver(nu_np, u1)
        state = sol.initial_state()
        ckpts = {0: state.clone()}
        for n in range(1, fam.nsteps + 1):
            sol.step_cn(state, fam.dt, 1, fam.tol, fam.restart, 20000)
            if n % fam.checkpoint == 0 and n < fam.nsteps:
                ckpts[n] = state.clone()
        ctx.fam, ctx.ckpts, ctx.nu_np, ctx.u1 = fam, ckpts, nu_np, u1
        sol.close()
        return state.clone()

    @staticmethod
    def backward(ctx, gL):
        fam, ckpts, nu_np, u1 = ctx.fam, ctx.ckpts, ctx.nu_np, ctx.u1
        t_enter = time.perf_counter()
        sol = fam.solver(nu_np, u1)
        lam = gL.detach().to(torch.float64).contiguous().clone()
        grads = sol.field_grad_buffers(lam.device, which=U1_FIELDS + ("nu",))
        end = fam.nsteps
        t_rec = t_adj = 0.0
        iters = []
        sync = torch.cuda.synchronize if lam.is_cuda else (lambda: None)  # wall-clock parts only
        sync()
        t_setup = time.perf_counter() - t_enter
        for s0 in reversed(sorted(ckpts)):
            # recompute the states of [s0, end] from the checkpoint
            t0 = time.perf_counter()
            states = [ckpts[s0].clone()]
            x = ckpts[s0].clone()
            for _ in range(s0, end):
                sol.step_cn(x, fam.dt, 1, fam.tol, fam.restart, 20000)
                states.append(x.clone())
            sync()
            t1 = time.perf_counter()
            for k in range(end - s0, 0, -1):
                st = sol.adjoint_step("cn", states[k - 1], states[k], lam, fam.dt, grads, fam.tol, fam.restart,
                                      20000)
                iters.append(int(st.iterations))
            t_rec += t1 - t0
            t_adj += time.perf_counter() - t1
            end = s0
        g_u1 = _chain_u1(grads, sol.field_arrays(fam.field_derivative(nu_np, u1)), lam.device)
        sol.close()
        fam.last_backward = {"total_s": time.perf_counter() - t_enter, "setup_s": t_setup,
                             "recompute_s": t_rec, "adjoint_s": t_adj,
                             "adjoint_iterations_per_step": sum(iters) / max(1, len(iters))}
        return grads["nu"], g_u1.cpu(), None


class ERKTrajectory(torch.autograd.Function):
    """zeta_N = RK4^N(zeta_0 = initial state; nu, U1).  Inputs: nu_nodes (npv, float64, cuda),
    U1 (0-d float64 tensor).  Returns the final state (N, float64, cuda)."""

    @staticmethod
    def forward(ctx, nu_nodes, U1, fam: CNProblemFamily):
        u1 = float(U1)
        nu_np = nu_nodes.detach().cpu().numpy()
        sol = fam.solver(nu_np, u1)
        state = sol.initial_state()
        ckpts = {0: state.clone()}
        for n in range(1, fam.nsteps + 1):
            sol.step_erk(state, fam.dt, 1)
            if n % fam.checkpoint == 0 and n < fam.nsteps:
                ckpts[n] = state.clone()
        ctx.fam, ctx.ckpts, ctx.nu_np, ctx.u1 = fam, ckpts, nu_np, u1
        sol.close()
        return state.clone()

    @staticmethod
    def backward(ctx, gL):
        fam, ckpts, nu_np, u1 = ctx.fam, ctx.ckpts, ctx.nu_np, ctx.u1
        sol = fam.solver(nu_np, u1)
        lam = gL.detach().to(torch.float64).contiguous().clone()
        grads = sol.field_grad_buffers(lam.device, which=U1_FIELDS + ("nu",))
        end = fam.nsteps
        for s0 in reversed(sorted(ckpts)):
            # the states that start the steps of [s0, end)
            states = [ckpts[s0].clone()]
            x = ckpts[s0].clone()
            for _ in range(s0, end - 1):
                sol.step_erk(x, fam.dt, 1)
                states.append(x.clone())
            for k in range(end - s0 - 1, -1, -1):
                sol.adjoint_step("erk4", states[k], None, lam, fam.dt, grads)
            end = s0
        g_u1 = _chain_u1(grads, sol.field_arrays(fam.field_derivative(nu_np, u1)), lam.device)
        sol.close()
        return grads["nu"], g_u1.cpu(), None


def spectrum_loss(state, prob, target, mask, x_range=(50.0, 150.0)):
    """L = sum_j (S_j - T_j)^2 over masked momentum cells j, with S_j = ln of the mean over the
    x-cells whose centre lies in x_range of the cell-averaged f_000 (shock workload layout)."""
    nx, npc = len(prob.edges[0]) - 1, len(prob.edges[1]) - 1
    nloc = (prob.k + 1) ** 2
    f = state.view(npc, nx, prob.n, nloc)[:, :, 0, :].mean(dim=2)  # Gauss weights equal for k <= 1
    xc = 0.5 * (prob.edges[0][1:] + prob.edges[0][:-1])
    sel = torch.from_numpy((xc > x_range[0]) & (xc < x_range[1])).to(state.device)
    S = torch.log(f[:, sel].mean(dim=1))
    m = torch.as_tensor(mask, device=state.device)
    return ((S - target.to(state.device)) ** 2)[m].sum()
