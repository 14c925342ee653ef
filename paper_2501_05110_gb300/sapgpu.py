"""Thin ctypes binding of the C ABI in include/sap.h (argument marshalling only).

Every step of the operator, the RK4 stages and the Crank--Nicolson / GMRES solve runs inside the
CUDA library ``libsapgpu.so``.  PyTorch supplies device memory and streams.  There is no CPU
fallback: loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libsapgpu.so")

SAP_OK, SAP_EINVAL, SAP_ENOMEM, SAP_ECUDA, SAP_ENOCONV, SAP_ETIMEOUT, SAP_EUNSUPPORTED = range(7)
AXIS = {"x": 0, "y": 1, "z": 2, "p": 3, "lnp": 4}
BC = {"periodic": 0, "inflow0": 1, "continuous": 2}
TERM = {"adv": 1, "mom": 2, "rot": 4, "coll": 8, "src": 16}
PREC = {"fp64": 0, "fp32": 1}
FLUX = {"upwind": 0, "llf": 1}
APPLY_D, APPLY_RHS, APPLY_T = 0, 1, 2
PTS_SPATIAL, PTS_FACE_X, PTS_FACE_Y, PTS_FACE_Z, PTS_PHASE = range(5)

SCHEME = {"erk4": 0, "cn": 1}
KERNEL = {"auto": 0, "rows": 1}
EXPORTS = ["sap_create", "sap_create_batch", "sap_batch_instance", "sap_field_points", "sap_set_fields", "sap_num_dofs", "sap_apply_operator",
           "sap_step_erk", "sap_step_erk_noalloc", "sap_step_cn", "sap_adjoint_step_cn", "sap_adjoint_step_erk",
           "sap_adjoint_step", "sap_step_theta", "sap_set_fields_device", "sap_set_flux", "sap_probe_fma", "sap_apply_cost", "sap_destroy", "sap_last_error", "sap_coupling_matrix",
           "sap_set_apply_kernel", "sap_apply_kernel_in_use"]
# field arrays of sap_set_fields / gradient arrays of sap_adjoint_step, in struct order
FIELDS = ("U", "gradU", "DUDt", "Bw", "Uface0", "Uface1", "Uface2", "nu", "s000")


class SapError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"sap status {status}: {msg}")
        self.status = status


class Desc(C.Structure):
    _fields_ = [("ndim", C.c_int), ("axis_kind", C.c_int * 3), ("ncells", C.c_int * 3),
                ("edges", C.POINTER(C.c_double) * 3), ("bc_lo", C.c_int * 3), ("bc_hi", C.c_int * 3),
                ("lmax", C.c_int), ("degree", C.c_int), ("V", C.c_double), ("terms", C.c_uint)]


class SolverStats(C.Structure):
    _fields_ = [("steps", C.c_int), ("iterations", C.c_int64), ("max_iterations", C.c_int),
                ("last_rel_residual", C.c_double), ("kernel_launches", C.c_int64)]


class FieldGrads(C.Structure):
    _fields_ = [("U", C.c_void_p), ("gradU", C.c_void_p), ("DUDt", C.c_void_p), ("Bw", C.c_void_p),
                ("Uface", C.c_void_p * 3), ("nu", C.c_void_p), ("s000", C.c_void_p)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libsapgpu.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = C.CDLL(path)
    vp, i64p, dp = C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double)
    lib.sap_create.argtypes = [C.POINTER(Desc), C.c_int, C.POINTER(C.c_void_p)]
    lib.sap_create_batch.argtypes = [C.c_int, C.POINTER(Desc), C.c_int, C.POINTER(C.c_void_p)]
    lib.sap_batch_instance.argtypes = [vp, C.c_int, C.POINTER(C.c_void_p), i64p]
    lib.sap_field_points.argtypes = [vp, C.c_int, dp, i64p]
    lib.sap_set_fields.argtypes = [vp, dp, dp, dp, dp, C.POINTER(dp), dp, dp]
    lib.sap_set_fields_device.argtypes = [vp, vp, vp, vp, vp, C.POINTER(vp), vp, vp, vp]
    lib.sap_set_flux.argtypes = [vp, C.c_int]
    lib.sap_set_apply_kernel.argtypes = [vp, C.c_int, C.c_int]
    lib.sap_apply_kernel_in_use.argtypes = [vp, C.POINTER(C.c_int)]
    lib.sap_num_dofs.argtypes = [vp, i64p]
    lib.sap_apply_operator.argtypes = [vp, vp, vp, C.c_int, vp]
    lib.sap_step_erk.argtypes = [vp, vp, C.c_double, C.c_int, vp]
    lib.sap_step_erk_noalloc.argtypes = [vp, vp, C.c_double, C.c_int, vp]
    lib.sap_step_cn.argtypes = [vp, vp, C.c_double, C.c_int, C.c_double, C.c_int, C.c_int,
                                C.POINTER(SolverStats), vp]
    lib.sap_step_theta.argtypes = [vp, vp, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int, C.c_int,
                                   C.POINTER(SolverStats), vp]
    lib.sap_apply_cost.argtypes = [vp, dp, dp]
    lib.sap_probe_fma.argtypes = [C.c_int, dp]
    lib.sap_adjoint_step_cn.argtypes = [vp, vp, vp, vp, C.c_double, C.c_double, C.c_int, C.c_int, vp, vp,
                                        C.POINTER(SolverStats), vp]
    lib.sap_adjoint_step_erk.argtypes = [vp, vp, vp, C.c_double, vp, vp, C.POINTER(SolverStats), vp]
    lib.sap_adjoint_step.argtypes = [vp, C.c_int, vp, vp, vp, C.c_double, C.c_double, C.c_int, C.c_int,
                                     C.POINTER(FieldGrads), C.POINTER(SolverStats), vp]
    lib.sap_destroy.argtypes = [vp]
    lib.sap_last_error.argtypes = [vp]
    lib.sap_last_error.restype = C.c_char_p
    lib.sap_coupling_matrix.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp]
    for name in EXPORTS:
        getattr(lib, name).restype = C.c_int if name != "sap_last_error" else C.c_char_p
    _lib = lib
    return lib


def coupling_matrix(lmax: int, which: int, a: int = 0, b: int = 0) -> np.ndarray:
    """The library's host-built n x n coupling matrix (see sap_coupling_matrix)."""
    lib = load_library()
    n = (lmax + 1) ** 2
    out = np.zeros(n * n)
    st = lib.sap_coupling_matrix(lmax, which, a, b, out.ctypes.data_as(C.POINTER(C.c_double)))
    if st != SAP_OK:
        raise SapError(st, "sap_coupling_matrix")
    return out.reshape(n, n)


def probe_fma(precision: str = "fp64") -> float:
    """Measured FMA throughput (flop/s) of the current device (sap_probe_fma)."""
    lib = load_library()
    v = C.c_double()
    st = lib.sap_probe_fma(PREC[precision], C.byref(v))
    if st != SAP_OK:
        raise SapError(st, "sap_probe_fma")
    return v.value


def _dptr(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def make_desc(prob):
    """sap_desc for a workloads.Problem; returns (desc, keep-alive edge arrays)."""
    D = len(prob.axes)
    d = Desc()
    d.ndim = D
    edges = [np.ascontiguousarray(e, dtype=np.float64) for e in prob.edges]
    for a in range(D):
        d.axis_kind[a] = AXIS[prob.axes[a]]
        d.ncells[a] = len(edges[a]) - 1
        d.edges[a] = edges[a].ctypes.data_as(C.POINTER(C.c_double))
        d.bc_lo[a] = BC[prob.bc[a][0]]
        d.bc_hi[a] = BC[prob.bc[a][1]]
    d.lmax, d.degree, d.V = prob.lmax, prob.k, float(prob.V)
    d.terms = sum(TERM[t] for t in prob.terms)
    return d, edges


class Solver:
    """One problem on the current CUDA device (wraps a sap_handle)."""

    def __init__(self, prob, precision: str = "fp64", handle=None):
        self.lib = load_library()
        self.prob = prob
        self.precision = precision
        self.owned = handle is None
        if handle is None:
            d, self._edges = make_desc(prob)
            h = C.c_void_p()
            st = self.lib.sap_create(C.byref(d), PREC[precision], C.byref(h))
            if st != SAP_OK:
                raise SapError(st, self.lib.sap_last_error(None).decode())
            self.h = h
        else:
            self.h = handle
        n = C.c_int64()
        self._check(self.lib.sap_num_dofs(self.h, C.byref(n)))
        self.N = n.value
        if getattr(prob, "flux", "upwind") != "upwind":
            self._check(self.lib.sap_set_flux(self.h, FLUX[prob.flux]))
        self.set_fields(prob)

    # -- helpers -------------------------------------------------------------------------------
    def _check(self, st):
        if st != SAP_OK:
            raise SapError(st, self.lib.sap_last_error(self.h).decode())

    def points(self, which: int) -> np.ndarray:
        cnt = C.c_int64()
        self._check(self.lib.sap_field_points(self.h, which, None, C.byref(cnt)))
        if cnt.value == 0:
            return np.zeros((0, 0))
        dim = len(self.prob.axes) if which == PTS_PHASE else len([a for a in self.prob.axes if a in "xyz"])
        out = np.zeros((cnt.value, dim))
        self._check(self.lib.sap_field_points(self.h, which, _dptr(out), C.byref(cnt)))
        return out

    def _phase_xs_p(self, pts):
        prob = self.prob
        sp = [i for i, a in enumerate(prob.axes) if a in "xyz"]
        xs = pts[:, sp]
        p = None
        if prob.momentum is not None:
            col = pts[:, len(prob.axes) - 1]
            p = np.exp(col) if prob.momentum == "lnp" else col
        return xs, p

    def field_arrays(self, prob) -> dict:
        """The problem's fields at the library's points, in the layouts of sap_set_fields: U (nsv*3),
        gradU (nsv*9), DUDt (nsv*3), Bw (nsv*3), Uface0..2 (nsf_a, None for absent axes), nu and s000
        (npv)."""
        xs = self.points(PTS_SPATIAL)
        nsv = xs.shape[0]
        out = {"U": prob.U(xs), "gradU": prob.gradU(xs), "DUDt": prob.DUDt(xs),
               "Bw": prob.B(xs) if prob.momentum is not None else prob.omega(xs)}
        for k, width in (("U", 3), ("gradU", 9), ("DUDt", 3), ("Bw", 3)):
            out[k] = np.ascontiguousarray(out[k], dtype=np.float64).reshape(nsv * width)
        for a in range(3):
            fp = self.points(PTS_FACE_X + a)
            out[f"Uface{a}"] = np.ascontiguousarray(prob.U(fp)[:, a], dtype=np.float64) if fp.shape[0] else None
        ph = self.points(PTS_PHASE)
        pxs, pp = self._phase_xs_p(ph)
        out["nu"] = np.ascontiguousarray(prob.nu(pxs, pp), dtype=np.float64)
        out["s000"] = np.ascontiguousarray(prob.s000(pxs, pp), dtype=np.float64)
        return out

    def set_fields(self, prob):
        """Evaluate the problem's fields at the library's points and upload them."""
        f = self.field_arrays(prob)
        face_ptrs = (C.POINTER(C.c_double) * 3)(*[_dptr(f[f"Uface{a}"]) for a in range(3)])
        self._check(self.lib.sap_set_fields(self.h, _dptr(f["U"]), _dptr(f["gradU"]), _dptr(f["DUDt"]),
                                            _dptr(f["Bw"]), face_ptrs, _dptr(f["nu"]), _dptr(f["s000"])))

    def set_fields_device(self, fields: dict, stream=None):
        """sap_set_fields_device from device tensors (keys of FIELDS; missing or None: not given)."""
        ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        faces = (C.c_void_p * 3)(*[ptr(fields.get(f"Uface{a}")) for a in range(3)])
        self._check(self.lib.sap_set_fields_device(self.h, ptr(fields.get("U")), ptr(fields.get("gradU")),
                                                   ptr(fields.get("DUDt")), ptr(fields.get("Bw")), faces,
                                                   ptr(fields.get("nu")), ptr(fields.get("s000")),
                                                   _stream_handle(stream)))

    def initial_state(self, device="cuda"):
        """Nodal values of f^0 at the phase-space nodes, canonical layout, FP64 torch tensor."""
        import torch
        ph = self.points(PTS_PHASE)
        f0 = np.asarray(self.prob.f0(ph), dtype=np.float64)  # (ncell*nloc, n)
        nloc = (self.prob.k + 1) ** len(self.prob.axes)
        ncell = ph.shape[0] // nloc
        y = f0.reshape(ncell, nloc, self.prob.n).transpose(0, 2, 1).reshape(-1)
        return torch.from_numpy(np.ascontiguousarray(y)).to(device)

    # -- compute -------------------------------------------------------------------------------
    def apply(self, x, y, mode: int = APPLY_D, stream=None):
        self._check(self.lib.sap_apply_operator(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                                mode, _stream_handle(stream)))
        return y

    def step_erk(self, state, dt: float, nsteps: int, stream=None):
        self._check(self.lib.sap_step_erk(self.h, C.c_void_p(state.data_ptr()), dt, nsteps, _stream_handle(stream)))
        return state

    def step_erk_noalloc(self, state, dt: float, nsteps: int, stream=None):
        """RK4 steps that allocate no device memory (stage buffers in the library's fixed array)."""
        self._check(self.lib.sap_step_erk_noalloc(self.h, C.c_void_p(state.data_ptr()), dt, nsteps,
                                                  _stream_handle(stream)))
        return state

    def step_cn(self, state, dt: float, nsteps: int, tol: float = 1e-10, restart: int = 30, maxit: int = 2000,
                stream=None) -> SolverStats:
        st = SolverStats()
        self._check(self.lib.sap_step_cn(self.h, C.c_void_p(state.data_ptr()), dt, nsteps, tol, restart, maxit,
                                         C.byref(st), _stream_handle(stream)))
        return st

    def step_theta(self, state, dt: float, theta: float, nsteps: int, tol: float = 1e-10, restart: int = 30,
                   maxit: int = 2000, stream=None) -> SolverStats:
        """theta-method steps (0 forward Euler, 1 backward Euler, 1/2 Crank--Nicolson)."""
        st = SolverStats()
        self._check(self.lib.sap_step_theta(self.h, C.c_void_p(state.data_ptr()), dt, theta, nsteps, tol, restart,
                                            maxit, C.byref(st), _stream_handle(stream)))
        return st

    def adjoint_step_cn(self, zeta_prev, zeta_next, lam, dt: float, tol: float = 1e-12, restart: int = 30,
                        maxit: int = 4000, mu_out=None, grad_nu=None, stream=None) -> SolverStats:
        """lam <- dJ/dzeta_prev given dJ/dzeta_next (in place); optional mu and nodal nu-gradient."""
        st = SolverStats()
        ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        self._check(self.lib.sap_adjoint_step_cn(self.h, ptr(zeta_prev), ptr(zeta_next), ptr(lam), dt, tol, restart,
                                                 maxit, ptr(mu_out), ptr(grad_nu), C.byref(st),
                                                 _stream_handle(stream)))
        return st

    def adjoint_step_erk(self, zeta_prev, lam, dt: float, grad_nu=None, stages_out=None,
                         stream=None) -> SolverStats:
        """lam <- dJ/dzeta_prev given dJ/dzeta_next (in place) for the RK4 step from zeta_prev;
        optional nodal nu-gradient and the stage inputs / stage adjoints (7 N doubles)."""
        st = SolverStats()
        ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        self._check(self.lib.sap_adjoint_step_erk(self.h, ptr(zeta_prev), ptr(lam), dt, ptr(grad_nu),
                                                  ptr(stages_out), C.byref(st), _stream_handle(stream)))
        return st

    def field_grad_buffers(self, device="cuda", which=FIELDS) -> dict:
        """Zeroed FP64 device accumulators for sap_adjoint_step, one per field array (shapes of
        field_arrays; absent face axes are None)."""
        import torch
        shapes = {k: (None if v is None else v.size) for k, v in self.field_arrays(self.prob).items()}
        return {k: (None if shapes[k] is None else torch.zeros(shapes[k], dtype=torch.float64, device=device))
                for k in which}

    def adjoint_step(self, scheme: str, zeta_prev, zeta_next, lam, dt: float, grads: dict = None,
                     tol: float = 1e-12, restart: int = 30, maxit: int = 4000, stream=None) -> SolverStats:
        """sap_adjoint_step: lam <- dJ/dzeta_prev (in place) and dJ/d(field) added into the device
        tensors of ``grads`` (keys of FIELDS; missing keys or None: not formed)."""
        st = SolverStats()
        ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        g = FieldGrads()
        grads = grads or {}
        for k in ("U", "gradU", "DUDt", "Bw", "nu", "s000"):
            setattr(g, k, ptr(grads.get(k)))
        for a in range(3):
            g.Uface[a] = ptr(grads.get(f"Uface{a}"))
        self._check(self.lib.sap_adjoint_step(self.h, SCHEME[scheme], ptr(zeta_prev), ptr(zeta_next), ptr(lam),
                                              dt, tol, restart, maxit, C.byref(g), C.byref(st),
                                              _stream_handle(stream)))
        return st

    def set_apply_kernel(self, kernel="auto", cells_per_block=0):
        """Choose the forward apply's kernel: "auto" (the node kernel where the problem has uniform
        coefficients, 3-D, k = 2, l_max <= 5) or "rows"."""
        self._check(self.lib.sap_set_apply_kernel(self.h, KERNEL[kernel], int(cells_per_block)))

    def apply_kernel_in_use(self):
        """"node" or "rows" (the kernel the forward apply runs now)."""
        u = C.c_int()
        self._check(self.lib.sap_apply_kernel_in_use(self.h, C.byref(u)))
        return "node" if u.value else "rows"

    def apply_cost(self):
        """(flops, bytes) of one operator apply, from the library's cost model."""
        f, b = C.c_double(), C.c_double()
        self._check(self.lib.sap_apply_cost(self.h, C.byref(f), C.byref(b)))
        return f.value, b.value

    def close(self):
        if getattr(self, "h", None) and self.owned:
            self.lib.sap_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch(Solver):
    """Independent problems run together (sap_create_batch): one launch per operator apply over all
    instances, lock-step per-instance GMRES.  The state is the concatenation of the instances'
    canonical states (``offsets``)."""

    def __init__(self, probs, precision: str = "fp32"):
        self.lib = load_library()
        self.probs = list(probs)
        self.precision = precision
        self.owned = True
        descs = (Desc * len(self.probs))()
        self._edges = []
        for i, p in enumerate(self.probs):
            d, e = make_desc(p)
            descs[i] = d
            self._edges.append(e)
        h = C.c_void_p()
        st = self.lib.sap_create_batch(len(self.probs), descs, PREC[precision], C.byref(h))
        if st != SAP_OK:
            raise SapError(st, self.lib.sap_last_error(None).decode())
        self.h = h
        self.instances, self.offsets = [], []
        for i, p in enumerate(self.probs):
            sub, off = C.c_void_p(), C.c_int64()
            self._check(self.lib.sap_batch_instance(self.h, i, C.byref(sub), C.byref(off)))
            self.instances.append(Solver(p, precision, handle=sub))
            self.offsets.append(off.value)
        n = C.c_int64()
        self._check(self.lib.sap_num_dofs(self.h, C.byref(n)))
        self.N = n.value

    def initial_state(self, device="cuda"):
        import torch
        return torch.cat([s.initial_state(device) for s in self.instances])

    def split(self, v):
        """Views of a batch vector per instance."""
        return [v[o:o + s.N] for o, s in zip(self.offsets, self.instances)]
