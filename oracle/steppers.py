"""Time stepping of the semi-discrete system M zeta' + D zeta = h.

TEST INFRASTRUCTURE ONLY: part of the FP64 CPU oracle (see ``oracle/__init__.py``).

* classical explicit fourth-order Runge--Kutta (ERK4, Sec. 3.4, last paragraph);
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
