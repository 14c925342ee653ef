"""Build and call the oracle's multi-threaded C driver (csr_driver.c).

TEST INFRASTRUCTURE ONLY: part of the FP64 CPU oracle.  It times the oracle's assembled
Crank--Nicolson and RK4 steps on all host cores for the CPU baselines (bench.py) and is checked
against the oracle's Python steppers in tests/.  The library never uses it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csr_driver.c")
LIB = os.path.join(HERE, "_lib", "liboracle_csr.so")


def build(force: bool = False) -> str:
    """gcc -O2 -fopenmp -shared: no architecture-specific flags (the same source builds on x86 and Arm)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", LIB + ".tmp", SRC, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gcc failed for {SRC}:\n{r.stdout}\n{r.stderr}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        p = C.c_void_p
        lib.oracle_cn_gmres_steps.argtypes = [C.c_int64, p, p, p, p, p, p, p, p, C.c_int, C.c_double, C.c_int,
                                              C.c_int, C.c_int, C.POINTER(C.c_int64)]
        lib.oracle_cn_gmres_steps.restype = C.c_int
        lib.oracle_rk4_steps.argtypes = [C.c_int64, C.c_int, C.c_int, p, p, p, p, p, p, C.c_int, C.c_double, C.c_int]
        lib.oracle_rk4_steps.restype = C.c_int
        _lib = lib
    return _lib


class CNDriver:
    """The oracle's CN step A z' = B z + dt h (A = M + dt/2 D, B = M - dt/2 D) for one assembled
    discretisation, solved by the C driver's GMRES on all OpenMP threads."""

    def __init__(self, disc, dt: float):
        A = (disc.M + 0.5 * dt * disc.D).tocsr()
        B = (disc.M - 0.5 * dt * disc.D).tocsr()
        self.N = disc.N
        self._keep = []
        self.A = self._csr(A)
        self.B = self._csr(B)
        self.dth = np.ascontiguousarray(dt * disc.h, dtype=np.float64)

    def _csr(self, m):
        m.sort_indices()
        rp = np.ascontiguousarray(m.indptr, dtype=np.int64)
        ci = np.ascontiguousarray(m.indices, dtype=np.int32)
        v = np.ascontiguousarray(m.data, dtype=np.float64)
        self._keep += [rp, ci, v]
        return rp, ci, v

    def steps(self, z, nsteps: int, tol=1e-10, restart=30, maxit=10000, threads=0):
        """Advances z (float64 array, in place) on `threads` OpenMP threads (0: all host cores);
        returns (threads used, GMRES iterations)."""
        lib = _load()
        its = C.c_int64()
        ptr = lambda a: C.c_void_p(a.ctypes.data)
        nt = lib.oracle_cn_gmres_steps(self.N, ptr(self.A[0]), ptr(self.A[1]), ptr(self.A[2]), ptr(self.B[0]),
                                       ptr(self.B[1]), ptr(self.B[2]), ptr(self.dth), ptr(z), nsteps, tol,
                                       restart, maxit, threads, C.byref(its))
        if nt < 0:
            raise MemoryError("oracle C driver: allocation failed")
        return nt, its.value


class RK4Driver:
    """The oracle's RK4 step on zeta' = M^-1 (h - D zeta) for one fully assembled discretisation,
    with the inverses of the mass blocks (one per cell, shared by the cell's coefficient rows)."""

    def __init__(self, disc):
        m = disc.D.tocsr()
        m.sort_indices()
        self.rp = np.ascontiguousarray(m.indptr, dtype=np.int64)
        self.ci = np.ascontiguousarray(m.indices, dtype=np.int32)
        self.v = np.ascontiguousarray(m.data, dtype=np.float64)
        self.minv = np.ascontiguousarray(np.linalg.inv(disc.mass_blocks), dtype=np.float64)
        self.h = np.ascontiguousarray(disc.h, dtype=np.float64)
        self.ncell, self.n, self.nloc = disc.mass_blocks.shape[0], disc.n, disc.mesh.nloc
        self.N = disc.N

    def steps(self, z, dt: float, nsteps: int, threads=0):
        """Advances z (float64, in place); returns the number of OpenMP threads used."""
        lib = _load()
        ptr = lambda a: C.c_void_p(a.ctypes.data)
        nt = lib.oracle_rk4_steps(self.ncell, self.n, self.nloc, ptr(self.rp), ptr(self.ci), ptr(self.v),
                                  ptr(self.minv), ptr(self.h), ptr(z), nsteps, dt, threads)
        if nt < 0:
            raise MemoryError("oracle C driver: allocation failed")
        return nt
