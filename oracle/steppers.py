"""Time stepping of the semi-discrete system M zeta' + D zeta = h.

TEST INFRASTRUCTURE ONLY: part of the FP64 CPU oracle (see ``oracle/__init__.py``).

* classical explicit fourth-order Runge--Kutta (ERK4, Sec. 3.4, last paragraph), its
  tangent-linear trajectory and the transpose of one step (for the discrete adjoint);
* the theta-method (M + dt theta D) zeta^n = (M - dt (1-theta) D) zeta^(n-1) + dt h
  (Eq. theta-method, Eq. system-matrix-rhs) with a time-independent D and h; theta = 0, 1, 1/2
  give forward Euler, backward Euler and Crank--Nicolson.  The linear system is solved exactly by a
  sparse LU factorisation (the paper only says it is solved iteratively, which changes the
  solution by at most the solver tolerance);
* restarted GMRES with right point-Jacobi preconditioning, used only as an iteration-count
  reference for the iterative solve.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def rk4(M, D, h, zeta0, dt, nsteps, callback=None):
    """Classical RK4 on zeta' = M^-1 (h - D zeta)."""
    Mlu = spla.splu(sp.csc_matrix(M))
    F = lambda z: Mlu.solve(h - D @ z)
    z = np.array(zeta0, dtype=float)
    for i in range(nsteps):
        k1 = F(z)
        k2 = F(z + 0.5 * dt * k1)
        k3 = F(z + 0.5 * dt * k2)
        k4 = F(z + dt * k3)
        z = z + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        if callback is not None:
            callback(i + 1, z)
    return z


def rk4_tangent(M, D, h, dD, zeta0, dt, nsteps):
    """Tangent of the RK4 trajectory (Sec. 3.4) along a parameter direction with dD = dD/dtheta.
    Each stage derivative k_i = F(Y_i), F(z) = M^-1 (h - D z), has the tangent
    dk_i = -M^-1 (dD Y_i + D dY_i), with dY_1 = d, dY_2 = d + dt/2 dk_1, dY_3 = d + dt/2 dk_2,
    dY_4 = d + dt dk_3, and the step gives d <- d + dt/6 (dk_1 + 2 dk_2 + 2 dk_3 + dk_4), d^0 = 0.
    Returns (z^N, d^N)."""
    Mlu = spla.splu(sp.csc_matrix(M))
    F = lambda z: Mlu.solve(h - D @ z)
    dF = lambda z, dz: -Mlu.solve(dD @ z + D @ dz)
    z = np.array(zeta0, dtype=float)
    d = np.zeros_like(z)
    for _ in range(nsteps):
        Y1, dY1 = z, d
        k1, dk1 = F(Y1), dF(Y1, dY1)
        Y2, dY2 = z + 0.5 * dt * k1, d + 0.5 * dt * dk1
        k2, dk2 = F(Y2), dF(Y2, dY2)
        Y3, dY3 = z + 0.5 * dt * k2, d + 0.5 * dt * dk2
        k3, dk3 = F(Y3), dF(Y3, dY3)
        Y4, dY4 = z + dt * k3, d + dt * dk3
        k4, dk4 = F(Y4), dF(Y4, dY4)
        z = z + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        d = d + dt / 6.0 * (dk1 + 2 * dk2 + 2 * dk3 + dk4)
    return z, d


def rk4_step_transpose(LT, dt, lam):
    """Transpose of the linear part of one RK4 step (Sec. 3.4).  For zeta' = s - L zeta with a
    constant operator L, the classical RK4 step maps zeta to R zeta + const, with R the stability
    polynomial sum_{j=0..4} (-dt L)^j / j!, so dJ/dzeta = R^T dJ/dzeta' = sum_j (-dt L^T)^j / j! lam.
    ``LT`` applies L^T; the sum is taken by Horner's rule:
    lam + (-dt L^T)(lam + (-dt L^T)/2 (lam + (-dt L^T)/3 (lam + (-dt L^T)/4 lam)))."""
    lam = np.asarray(lam, dtype=float)
    v = lam.copy()
    for j in (4, 3, 2, 1):
        v = lam + (-dt / j) * LT(v)
    return v


def theta_method(M, D, h, zeta0, dt, nsteps, theta=0.5, callback=None):
    """zeta^n from (M + dt theta D) zeta^n = (M - dt (1-theta) D) zeta^(n-1) + dt h."""
    lhs = spla.splu(sp.csc_matrix(M + dt * theta * D))
    rhs_op = M - dt * (1.0 - theta) * D
    z = np.array(zeta0, dtype=float)
    for i in range(nsteps):
        z = lhs.solve(rhs_op @ z + dt * h)
        if callback is not None:
            callback(i + 1, z)
    return z


def gmres(A, b, x0, tol=1e-10, restart=30, maxit=10000):
    """Restarted GMRES(restart), modified Gram--Schmidt Arnoldi, right preconditioned by the
    inverse diagonal of A.  Stops when ||b - A x|| <= tol ||b||.  Returns (x, iterations)."""
    A = sp.csr_matrix(A)
    dinv = 1.0 / A.diagonal()
    x = np.array(x0, dtype=float)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0
    its = 0
    while its < maxit:
        r = b - A @ x
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            break
        V = np.zeros((restart + 1, len(b)))
        H = np.zeros((restart + 1, restart))
        V[0] = r / beta
        g = np.zeros(restart + 1)
        g[0] = beta
        cs, sn = np.zeros(restart), np.zeros(restart)
        j_done = 0
        for j in range(restart):
            w = A @ (dinv * V[j])
            for i in range(j + 1):
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):  # apply previous Givens rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            if abs(g[j + 1]) <= tol * bnorm or its >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + dinv * (V[:j_done].T @ y)
    return x, its


def cn_tangent(M, D, h, dD, zeta0, dt, nsteps):
    """Tangent of the Crank--Nicolson trajectory along a parameter direction with dD = dD/dtheta:
    differentiating (M + dt/2 D) z^n = (M - dt/2 D) z^(n-1) + dt h (Eq. theta-method, theta = 1/2)
    gives (M + dt/2 D) d^n = (M - dt/2 D) d^(n-1) - dt/2 dD (z^n + z^(n-1)), d^0 = 0.
    Returns (z^N, d^N)."""
    lhs = spla.splu(sp.csc_matrix(M + 0.5 * dt * D))
    rhs_op = M - 0.5 * dt * D
    z = np.array(zeta0, dtype=float)
    d = np.zeros_like(z)
    for _ in range(nsteps):
        zn = lhs.solve(rhs_op @ z + dt * h)
        d = lhs.solve(rhs_op @ d - 0.5 * dt * (dD @ (zn + z)))
        z = zn
    return z, d
