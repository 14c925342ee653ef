"""Discrete adjoints of Crank--Nicolson and RK4 trajectories as torch.autograd.Functions.

The forward pass runs CN steps in the library (sap_step_cn) and keeps the state every
`checkpoint` steps.  The backward pass walks the segments from the end: it recomputes a segment's
states from its checkpoint and runs the library's adjoint step (sap_adjoint_step_cn) through them:
  A^T mu = lambda_n,   lambda_{n-1} = B^T mu,   dJ/dnu += -dt/2 mu . (dL/dnu)(zeta_{n-1} + zeta_n),
the last term being exact (nu enters the operator only through the pointwise collision term).  The
shock speed U1 enters through every field (U, grad U, dU/dt) and the upwind splits; its term
-dt/2 mu . (dL/dU1)(zeta_{n-1} + zeta_n) uses the operator's central difference in U1,
(L(U1 + e) - L(U1 - e)) / (2e) with e = 1e-6 U1, applied by the library.

RK4 (ERKTrajectory) follows the same pattern with the library's RK4 adjoint step
(sap_adjoint_step_erk): per step it recomputes the stage inputs Y_i, forms the stage adjoints kb_i
and returns lambda_{n-1} = R^T lambda_n (R the RK4 stability polynomial in -dt L) and the exact nu
term -sum_i kb_i . (dL/dnu) Y_i; the U1 term -sum_i kb_i . (dL/dU1) Y_i uses the same central
difference in U1 on the stage pairs the library hands back.  RK4 is explicit, so recomputed segments
reproduce the forward states exactly.

Only argument marshalling and the per-step bookkeeping live here; every operator apply, linear
solve and gradient accumulation runs in libsapgpu.so.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable

import numpy as np
import torch

from . import sapgpu


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
    u1_rel_eps: float = 1e-6
    # filled by the backward pass: wall time of its parts (s) and the adjoint GMRES iterations per step
    last_backward: dict = dataclasses.field(default_factory=dict)

    def solver(self, nu_nodes, U1):
        return sapgpu.Solver(self.make_problem(nu_nodes, U1), "fp64")


def _node_nu_problem(base_make, nu_nodes, U1):
    prob = base_make(U1)
    if nu_nodes is not None:
        vals = np.ascontiguousarray(nu_nodes, dtype=np.float64)
        prob.nu = lambda xs, p, _v=vals: _v
    return prob


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
        ctx.npv = nu_nodes.numel()
        sol.close()
        return state.clone()

    @staticmethod
    def backward(ctx, gL):
        fam, ckpts, nu_np, u1 = ctx.fam, ctx.ckpts, ctx.nu_np, ctx.u1
        t_enter = time.perf_counter()
        sol = fam.solver(nu_np, u1)
        eps = fam.u1_rel_eps * abs(u1)
        sol_p = fam.solver(nu_np, u1 + eps)
        sol_m = fam.solver(nu_np, u1 - eps)
        lam = gL.detach().to(torch.float64).contiguous().clone()
        grad_nu = torch.zeros(ctx.npv, dtype=torch.float64, device=lam.device)
        mu = torch.empty_like(lam)
        a = torch.empty_like(lam)
        b = torch.empty_like(lam)
        g_u1 = 0.0
        starts = sorted(ckpts)
        end = fam.nsteps
        t_rec = t_adj = 0.0
        iters = []
        sync = torch.cuda.synchronize if lam.is_cuda else (lambda: None)  # wall-clock parts only
        sync()
        t_setup = time.perf_counter() - t_enter
        for s0 in reversed(starts):
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
                zp, zn = states[k - 1], states[k]
                st = sol.adjoint_step_cn(zp, zn, lam, fam.dt, fam.tol, fam.restart, 20000, mu_out=mu,
                                         grad_nu=grad_nu)
                iters.append(int(st.iterations))
                w = zp + zn
                sol_p.apply(w, a)
                sol_m.apply(w, b)
                g_u1 += -0.5 * fam.dt * float(mu @ (a - b)) / (2 * eps)
            t_rec += t1 - t0
            t_adj += time.perf_counter() - t1
            end = s0
        for s in (sol, sol_p, sol_m):
            s.close()
        fam.last_backward = {"total_s": time.perf_counter() - t_enter, "setup_s": t_setup,
                             "recompute_s": t_rec, "adjoint_s": t_adj,
                             "adjoint_iterations_per_step": sum(iters) / max(1, len(iters))}
        return grad_nu, torch.tensor(g_u1, dtype=torch.float64), None


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
        ctx.npv = nu_nodes.numel()
        sol.close()
        return state.clone()

    @staticmethod
    def backward(ctx, gL):
        fam, ckpts, nu_np, u1 = ctx.fam, ctx.ckpts, ctx.nu_np, ctx.u1
        sol = fam.solver(nu_np, u1)
        eps = fam.u1_rel_eps * abs(u1)
        sol_p = fam.solver(nu_np, u1 + eps)
        sol_m = fam.solver(nu_np, u1 - eps)
        lam = gL.detach().to(torch.float64).contiguous().clone()
        N = lam.numel()
        grad_nu = torch.zeros(ctx.npv, dtype=torch.float64, device=lam.device)
        stages = torch.empty(7 * N, dtype=torch.float64, device=lam.device)
        a = torch.empty_like(lam)
        b = torch.empty_like(lam)
        g_u1 = torch.zeros((), dtype=torch.float64, device=lam.device)
        end = fam.nsteps
        for s0 in reversed(sorted(ckpts)):
            # the states that start the steps of [s0, end)
            states = [ckpts[s0].clone()]
            x = ckpts[s0].clone()
            for _ in range(s0, end - 1):
                sol.step_erk(x, fam.dt, 1)
                states.append(x.clone())
            for k in range(end - s0 - 1, -1, -1):
                y = states[k]
                sol.adjoint_step_erk(y, lam, fam.dt, grad_nu=grad_nu, stages_out=stages)
                Y = [y, stages[:N], stages[N:2 * N], stages[2 * N:3 * N]]
                for i in range(4):
                    kb = stages[(3 + i) * N:(4 + i) * N]
                    sol_p.apply(Y[i], a)
                    sol_m.apply(Y[i], b)
                    g_u1 -= kb @ (a - b) / (2 * eps)
            end = s0
        for s in (sol, sol_p, sol_m):
            s.close()
        return grad_nu, g_u1.cpu(), None


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
