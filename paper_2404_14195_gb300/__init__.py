"""Python binding of librbfgb — the GB300 (sm_103a) meshless porous-media solvers
of arXiv 2404.14195 (RBF-FD stencils and weights, the artificial-compressibility
Navier-Stokes step, the TRT meshless lattice Boltzmann step, permeability and
drag).

Argument marshalling only: every call goes through the C ABI declared in
``include/rbfgb.h`` and every step of the method runs in the library's CUDA
kernels.  There is no CPU fallback: importing works anywhere, but creating a
``Solver`` raises ``RbfError`` when the CUDA library is missing or no GPU is
usable.

The ``rbf_*`` names of the C ABI are exported as ctypes functions by ``lib()``;
``Solver`` wraps one ``rbf_ctx`` with numpy in and out.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

RBF_OK, RBF_EINVAL, RBF_ECUDA, RBF_ESINGULAR = 0, -1, -2, -3
RBF_EDIVERGED, RBF_ENOTCONVERGED, RBF_ETIMEOUT, RBF_ENOMEM = -4, -5, -6, -7
RBF_SOLVER_ACM, RBF_SOLVER_LBM = 0, 1
RBF_FP64, RBF_FP32, RBF_FP32C, RBF_FP32R = 0, 1, 2, 3
RBF_OP_DX, RBF_OP_DY, RBF_OP_DZ, RBF_OP_LAP, RBF_OP_LBM0 = 0, 1, 2, 3, 16

_ERRNAMES = {RBF_EINVAL: "EINVAL", RBF_ECUDA: "ECUDA", RBF_ESINGULAR: "ESINGULAR",
             RBF_EDIVERGED: "EDIVERGED", RBF_ENOTCONVERGED: "ENOTCONVERGED",
             RBF_ETIMEOUT: "ETIMEOUT", RBF_ENOMEM: "ENOMEM"}


class RbfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class rbf_weight_report(ctypes.Structure):
    _fields_ = [("n_systems", ctypes.c_int64), ("n_singular", ctypes.c_int64), ("h_min", ctypes.c_double)]


class rbf_params(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("nu", ctypes.c_double), ("g", ctypes.c_double * 3),
                ("rho", ctypes.c_double), ("dt", ctypes.c_double), ("cfl", ctypes.c_double),
                ("beta", ctypes.c_double), ("v_ref", ctypes.c_double), ("n_p", ctypes.c_int),
                ("tau_plus", ctypes.c_double), ("magic", ctypes.c_double)]


class rbf_tune_report(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("n_candidates", ctypes.c_int), ("code", ctypes.c_int * 16),
                ("ms_per_step", ctypes.c_double * 16), ("chosen", ctypes.c_int)]


class rbf_batch_cell_result(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("residual", ctypes.c_double), ("k_over_d2", ctypes.c_double),
                ("status", ctypes.c_int)]


class rbf_solve_opts(ctypes.Structure):
    _fields_ = [("max_steps", ctypes.c_int64), ("check_every", ctypes.c_int), ("tol", ctypes.c_double),
                ("m_p", ctypes.c_int)]


class rbf_solve_result(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("residual", ctypes.c_double), ("k_over_d2", ctypes.c_double),
                ("converged", ctypes.c_int)]


_lib = None
_lock = threading.Lock()

# C ABI: name -> (restype, argtypes)
_P, _I, _I64, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
ABI = {
    "rbf_create": (_I, [ctypes.POINTER(_P), _I, _P]),
    "rbf_destroy": (_I, [_P]),
    "rbf_last_error": (ctypes.c_char_p, [_P]),
    "rbf_set_nodes": (_I, [_P, _I64, _P, _P, _P]),
    "rbf_set_sphere": (_I, [_P, _P, _D]),
    "rbf_build_stencils": (_I, [_P, _I]),
    "rbf_get_stencils": (_I, [_P, _P]),
    "rbf_compute_weights": (_I, [_P, _I, _I, _I, _I, _D, ctypes.POINTER(rbf_weight_report)]),
    "rbf_get_weights": (_I, [_P, _I, _P]),
    "rbf_init": (_I, [_P, ctypes.POINTER(rbf_params)]),
    "rbf_step": (_I, [_P, _I]),
    "rbf_get_fields": (_I, [_P, _P]),
    "rbf_set_fields": (_I, [_P, _P]),
    "rbf_lbm_get_populations": (_I, [_P, _P]),
    "rbf_lbm_set_populations": (_I, [_P, _P]),
    "rbf_permeability": (_I, [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "rbf_drag": (_I, [_P, _I, _P, ctypes.POINTER(_D)]),
    "rbf_pointwise_difference": (_I, [_P, _P, _P, _P]),
    "rbf_time_step": (_I, [_P, ctypes.POINTER(_D)]),
    "rbf_lbm_set_unknown_rule": (_I, [_P, _I]),
    "rbf_lbm_get_unknown_mask": (_I, [_P, _P]),
    "rbf_solve": (_I, [_P, ctypes.POINTER(rbf_solve_opts), ctypes.POINTER(rbf_solve_result)]),
    "rbf_last_step_timing": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_I64)]),
    "rbf_launch_count": (_I64, [_P]),
    "rbf_profile_steps": (_I, [_P, _I, _P, ctypes.POINTER(_I)]),
    "rbf_set_kernel_variant": (_I, [_P, _I]),
    "rbf_permeability_static": (_I, [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "rbf_autotune": (_I, [_P, _I, ctypes.POINTER(rbf_tune_report)]),
    "rbf_autotune_persistent": (_I, [_P, _I, ctypes.POINTER(rbf_tune_report)]),
    "rbf_set_persistent_block": (_I, [_P, _I]),
    "rbf_set_wait_limit": (_I, [_P, _D]),
    "rbf_batch_autotune": (_I, [_P, _I, ctypes.POINTER(rbf_tune_report)]),
    "rbf_batch_create": (_I, [ctypes.POINTER(_P), _I, _P]),
    "rbf_batch_destroy": (_I, [_P]),
    "rbf_batch_last_error": (ctypes.c_char_p, [_P]),
    "rbf_batch_add_cell": (_I, [_P, _I64, _P, _P, _P, _P, _D, _I]),
    "rbf_batch_build": (_I, [_P, _I, _I, ctypes.POINTER(rbf_weight_report)]),
    "rbf_batch_init": (_I, [_P, ctypes.POINTER(rbf_params)]),
    "rbf_batch_solve": (_I, [_P, ctypes.POINTER(rbf_solve_opts), _P]),
    "rbf_batch_num_cells": (_I, [_P]),
    "rbf_batch_cell": (_P, [_P, _I]),
    "rbf_mlp_num_params": (_I64, []),
    "rbf_mlp_create": (_I, [ctypes.POINTER(_P), _I, _P]),
    "rbf_mlp_destroy": (_I, [_P]),
    "rbf_mlp_last_error": (ctypes.c_char_p, [_P]),
    "rbf_mlp_set_params": (_I, [_P, _P]),
    "rbf_mlp_get_params": (_I, [_P, _P]),
    "rbf_mlp_set_data": (_I, [_P, _I64, _P, _P, _P, _P]),
    "rbf_mlp_train": (_I, [_P, _I, _I, _D, ctypes.c_uint64, _P]),
    "rbf_mlp_gradient": (_I, [_P, _I, _P, _P, ctypes.POINTER(_D)]),
    "rbf_mlp_predict": (_I, [_P, _I64, _P, _P, _P, _P]),
    "rbf_mlp_warm_start": (_I, [_P, _P, _P]),
    "rbf_mlp_set_fused": (_I, [_P, _I]),
    "rbf_mlp_launch_count": (_I64, [_P]),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Load librbfgb.so (built in-tree by ``_build.build()``); raises if missing."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RbfError(RBF_ECUDA, f"CUDA library not built: {path} (run __graft_entry__.build())")
            L = ctypes.CDLL(path)
            for name, (res, args) in ABI.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _out(out, shape):
    """A float64 array of ``shape`` to receive a result: a new one, or the caller's
    ``out`` written in place (for instance a pinned host buffer, which the library's
    device-to-host copy then writes directly)."""
    if out is None:
        return np.empty(shape, np.float64)
    if (not isinstance(out, np.ndarray) or out.dtype != np.float64 or out.shape != tuple(shape)
            or not out.flags.c_contiguous or not out.flags.writeable):
        raise ValueError(f"out must be a writeable C-contiguous float64 array of shape {tuple(shape)}")
    return out


class Solver:
    """One case on one GPU: nodes, stencils, weights, fields (an ``rbf_ctx``)."""

    def __init__(self, device: int = 0, stream=None):
        L = lib()
        self._L = L
        h = ctypes.c_void_p()
        rc = L.rbf_create(ctypes.byref(h), device, stream)
        if rc != RBF_OK:
            raise RbfError(rc, "rbf_create failed (no usable CUDA device?)")
        self._h = h
        self.n = 0
        self.n_l = 0
        self.q = 0
        self.solver = None

    def close(self):
        if getattr(self, "_h", None):
            self._L.rbf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _ck(self, rc):
        if rc != RBF_OK:
            raise RbfError(rc, self._L.rbf_last_error(self._h).decode())
        return rc

    # -- nodes and geometry -------------------------------------------------
    def set_nodes(self, xyz, type_, normal=None):
        xyz = np.ascontiguousarray(xyz, np.float64)
        t = np.ascontiguousarray(type_, np.uint8)
        nrm = None if normal is None else np.ascontiguousarray(normal, np.float64)
        self._ck(self._L.rbf_set_nodes(self._h, len(xyz), _ptr(xyz), _ptr(t), None if nrm is None else _ptr(nrm)))
        self.n = len(xyz)

    def set_sphere(self, c, r):
        c = np.ascontiguousarray(c, np.float64)
        self._ck(self._L.rbf_set_sphere(self._h, _ptr(c), float(r)))

    def set_case(self, case):
        self.set_nodes(case["xyz"], case["type"], case["normal"])
        if case.get("centre") is not None and case.get("radius", 0) > 0:
            self.set_sphere(case["centre"], case["radius"])

    # -- stencils and weights ----------------------------------------------
    def build_stencils(self, n_l: int):
        self._ck(self._L.rbf_build_stencils(self._h, n_l))
        self.n_l = n_l

    def get_stencils(self):
        out = np.empty((self.n, self.n_l), np.int32)
        self._ck(self._L.rbf_get_stencils(self._h, _ptr(out)))
        return out

    def compute_weights(self, k: int = 3, m: int = 2, solver: int = RBF_SOLVER_ACM, q: int = 19, dx: float = 0.0):
        rep = rbf_weight_report()
        rc = self._L.rbf_compute_weights(self._h, k, m, solver, q, dx, ctypes.byref(rep))
        self._ck(rc)
        self.solver = solver
        self.q = q if solver == RBF_SOLVER_LBM else 0
        return dict(n_systems=rep.n_systems, n_singular=rep.n_singular, h_min=rep.h_min)

    def get_weights(self, op: int):
        out = np.empty((self.n, self.n_l), np.float64)
        self._ck(self._L.rbf_get_weights(self._h, op, _ptr(out)))
        return out

    # -- time stepping --------------------------------------------------------
    def init(self, precision=RBF_FP64, nu=1.0, g=(1.0, 0.0, 0.0), rho=1.0, dt=0.0, cfl=0.1, beta=10.0,
             v_ref=0.0, n_p=3, tau_plus=0.8, magic=3.0 / 16.0):
        p = rbf_params()
        p.precision = precision
        p.nu = nu
        p.g[0], p.g[1], p.g[2] = g
        p.rho, p.dt, p.cfl, p.beta, p.v_ref, p.n_p = rho, dt, cfl, beta, v_ref, n_p
        p.tau_plus, p.magic = tau_plus, magic
        self._ck(self._L.rbf_init(self._h, ctypes.byref(p)))

    def step(self, nsteps: int):
        self._ck(self._L.rbf_step(self._h, int(nsteps)))

    def get_fields(self, out=None):
        out = _out(out, (self.n, 4))
        self._ck(self._L.rbf_get_fields(self._h, _ptr(out)))
        return out

    def set_fields(self, uvwp):
        a = np.ascontiguousarray(uvwp, np.float64)
        assert a.shape == (self.n, 4)
        self._ck(self._L.rbf_set_fields(self._h, _ptr(a)))

    def lbm_get_populations(self, out=None):
        out = _out(out, (self.q, self.n))
        self._ck(self._L.rbf_lbm_get_populations(self._h, _ptr(out)))
        return out

    def lbm_set_populations(self, f):
        a = np.ascontiguousarray(f, np.float64)
        assert a.shape == (self.q, self.n)
        self._ck(self._L.rbf_lbm_set_populations(self._h, _ptr(a)))

    # -- outputs --------------------------------------------------------------
    def lbm_set_unknown_rule(self, rule: int):
        """0: e_k . n > 0 (default); 1: departure point inside the solid."""
        self._ck(self._L.rbf_lbm_set_unknown_rule(self._h, int(rule)))

    def lbm_get_unknown_mask(self):
        out = np.empty(self.n, np.uint32)
        self._ck(self._L.rbf_lbm_get_unknown_mask(self._h, _ptr(out)))
        return out

    def permeability(self, m_p: int = 32):
        k, q = ctypes.c_double(), ctypes.c_double()
        self._ck(self._L.rbf_permeability(self._h, m_p, ctypes.byref(k), ctypes.byref(q)))
        return k.value, q.value

    def permeability_static(self, m_p: int = 32):
        """As permeability(m_p) without any device allocation (static scratch);
        needs a prior permeability(m_p) call that built the probe set."""
        k, q = ctypes.c_double(), ctypes.c_double()
        self._ck(self._L.rbf_permeability_static(self._h, m_p, ctypes.byref(k), ctypes.byref(q)))
        return k.value, q.value

    def drag(self, m_p: int = 32):
        F = np.zeros(3)
        K = ctypes.c_double()
        self._ck(self._L.rbf_drag(self._h, m_p, _ptr(F), ctypes.byref(K)))
        return F, K.value

    def pointwise_difference(self, other: "Solver"):
        """(delta, dv) of Eq. pointwise_error with v_a = this context's velocity and
        v_b = other's, per node in the caller's order (delta NaN where v_b = 0)."""
        return pointwise_difference(self, other)

    def solve(self, max_steps: int, tol: float, check_every: int = 100, m_p: int = 32, raise_on_cap=False):
        o = rbf_solve_opts(max_steps, check_every, tol, m_p)
        r = rbf_solve_result()
        rc = self._L.rbf_solve(self._h, ctypes.byref(o), ctypes.byref(r))
        if rc not in (RBF_OK, RBF_ENOTCONVERGED) or (raise_on_cap and rc != RBF_OK):
            self._ck(rc)
        return dict(steps=r.steps, residual=r.residual, k_over_d2=r.k_over_d2, converged=bool(r.converged))

    def last_step_timing(self):
        t, k, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        self._ck(self._L.rbf_last_step_timing(self._h, ctypes.byref(t), ctypes.byref(k), ctypes.byref(n)))
        return t.value, k.value, n.value

    def profile_steps(self, nsteps: int):
        """Mean device time (ms) of one launch of each kernel class over nsteps
        eagerly launched steps (LBM: [fused step]; ACM: [predict, pressure,
        wall pressure, correct])."""
        ms = np.zeros(4)
        nc = ctypes.c_int()
        self._ck(self._L.rbf_profile_steps(self._h, int(nsteps), _ptr(ms), ctypes.byref(nc)))
        return ms[:nc.value].copy()

    def set_kernel_variant(self, variant: int):
        """LBM step schedule: 0 / 2 one node per thread (256 / 128 threads per
        block); 1 / 3 / 4 / 5 one population pair per warp, unrolled 5 / 3 / 6 / 2;
        6 / 7 one node per thread on the node-record layout (256 threads;
        registers capped for five blocks per SM); 8 / 9 as 6 with 128 / 64
        threads per block; 10 as 6 as a programmatic dependent launch.  The state is rewritten when the layout changes.
        ACM (after compute_weights for the ACM): threads per block (64, 128,
        256) + 1000 x lanes per node (2, 4; 0 for one) of the step sweeps."""
        self._ck(self._L.rbf_set_kernel_variant(self._h, int(variant)))

    def autotune(self, trial_steps: int = 50):
        """Time the candidate step schedules on this case and keep the fastest;
        the state is restored afterwards.  Returns {code: ms_per_step}, chosen."""
        r = rbf_tune_report()
        self._ck(self._L.rbf_autotune(self._h, int(trial_steps), ctypes.byref(r)))
        return {r.code[i]: r.ms_per_step[i] for i in range(r.n_candidates)}, r.chosen

    def set_persistent_block(self, code: int):
        """Persistent ACM driver schedule code: threads per block (32, 64, 128,
        256) + 1000 x lanes per node (2, 4, 8; 0 for one), or -8 / -16 for one
        cluster of 8 / 16 CTAs."""
        self._ck(self._L.rbf_set_persistent_block(self._h, int(code)))

    def set_wait_limit(self, seconds: float):
        """Wall-clock limit of one grid-barrier wait of the persistent ACM driver
        (default 2 s); a wait that runs out ends the solve with RBF_ETIMEOUT."""
        self._ck(self._L.rbf_set_wait_limit(self._h, float(seconds)))

    def autotune_persistent(self, trial_steps: int = 200):
        """ACM: time the persistent driver's block sizes on this case and keep the
        fastest for solve(); the state is restored afterwards.  Returns
        {threads per block: ms_per_step}, chosen."""
        r = rbf_tune_report()
        self._ck(self._L.rbf_autotune_persistent(self._h, int(trial_steps), ctypes.byref(r)))
        return {r.code[i]: r.ms_per_step[i] for i in range(r.n_candidates)}, r.chosen

    def time_step(self) -> float:
        """Physical time of one step (ACM delta t, or the LBM delta t)."""
        d = ctypes.c_double()
        self._ck(self._L.rbf_time_step(self._h, ctypes.byref(d)))
        return d.value

    def launch_count(self) -> int:
        return int(self._L.rbf_launch_count(self._h))


def pointwise_difference(a: Solver, b: Solver):
    """rbf_pointwise_difference: (delta, dv) of Eq. pointwise_error between two
    initialised contexts on the same nodes (paper: a = MLBM, b = MNS)."""
    n = a.n
    delta, dv = np.empty(n), np.empty(n)
    rc = a._L.rbf_pointwise_difference(a._h, b._h, _ptr(delta), _ptr(dv))
    if rc != RBF_OK:
        msg = a._L.rbf_last_error(a._h).decode() or a._L.rbf_last_error(b._h).decode()
        raise RbfError(rc, msg)
    return delta, dv


def _params(precision=RBF_FP64, nu=1.0, g=(1.0, 0.0, 0.0), rho=1.0, dt=0.0, cfl=0.1, beta=10.0, v_ref=0.0,
            n_p=3, tau_plus=0.8, magic=3.0 / 16.0):
    p = rbf_params()
    p.precision = precision
    p.nu = nu
    p.g[0], p.g[1], p.g[2] = g
    p.rho, p.dt, p.cfl, p.beta, p.v_ref, p.n_p = rho, dt, cfl, beta, v_ref, n_p
    p.tau_plus, p.magic = tau_plus, magic
    return p


class _BorrowedSolver(Solver):
    """A cell of a Batch seen as a Solver (the batch owns the context)."""

    def __init__(self, L, handle, n, n_l):
        self._L = L
        self._h = ctypes.c_void_p(handle)
        self.n, self.n_l, self.q, self.solver = n, n_l, 0, RBF_SOLVER_ACM

    def close(self):
        self._h = None


class Batch:
    """Many cells solved together: one weight launch, one persistent step launch."""

    def __init__(self, device: int = 0, stream=None):
        L = lib()
        self._L = L
        h = ctypes.c_void_p()
        rc = L.rbf_batch_create(ctypes.byref(h), device, stream)
        if rc != RBF_OK:
            raise RbfError(rc, "rbf_batch_create failed (no usable CUDA device?)")
        self._h = h
        self._cells = []

    def close(self):
        if getattr(self, "_h", None):
            self._L.rbf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, rc, ok=(RBF_OK,)):
        if rc not in ok:
            raise RbfError(rc, self._L.rbf_batch_last_error(self._h).decode())
        return rc

    def add_cell(self, case, n_l: int):
        x = np.ascontiguousarray(case["xyz"], np.float64)
        t = np.ascontiguousarray(case["type"], np.uint8)
        nr = np.ascontiguousarray(case["normal"], np.float64)
        c = np.ascontiguousarray(case["centre"], np.float64)
        rc = self._L.rbf_batch_add_cell(self._h, len(x), _ptr(x), _ptr(t), _ptr(nr), _ptr(c), float(case["radius"]), n_l)
        if rc < 0:
            self._ck(rc)
        self._cells.append((len(x), n_l))
        return rc

    def build(self, k: int = 3, m: int = 2):
        rep = rbf_weight_report()
        self._ck(self._L.rbf_batch_build(self._h, k, m, ctypes.byref(rep)))
        return dict(n_systems=rep.n_systems, n_singular=rep.n_singular, h_min=rep.h_min)

    def init(self, **kw):
        p = _params(**kw)
        self._ck(self._L.rbf_batch_init(self._h, ctypes.byref(p)))

    def solve(self, max_steps: int, tol: float, check_every: int = 100, m_p: int = 32):
        o = rbf_solve_opts(max_steps, check_every, tol, m_p)
        res = (rbf_batch_cell_result * len(self._cells))()
        self._ck(self._L.rbf_batch_solve(self._h, ctypes.byref(o), res), ok=(RBF_OK, RBF_ENOTCONVERGED))
        return [dict(steps=r.steps, residual=r.residual, k_over_d2=r.k_over_d2, status=r.status) for r in res]

    def set_persistent_block(self, code: int):
        """Persistent-driver schedule code for every cell (see Solver.set_persistent_block)."""
        for i in range(len(self._cells)):
            self.cell(i).set_persistent_block(code)

    def autotune(self, trial_steps: int = 100):
        """Time the persistent driver's block sizes over all cells and keep the
        fastest; the cells' state is restored afterwards."""
        r = rbf_tune_report()
        self._ck(self._L.rbf_batch_autotune(self._h, int(trial_steps), ctypes.byref(r)))
        return {r.code[i]: r.ms_per_step[i] for i in range(r.n_candidates)}, r.chosen

    def cell(self, i: int) -> Solver:
        h = self._L.rbf_batch_cell(self._h, i)
        if not h:
            raise RbfError(RBF_EINVAL, "no such cell")
        n, n_l = self._cells[i]
        return _BorrowedSolver(self._L, h, n, n_l)


class Mlp:
    """The warm-start network (an ``rbf_mlp``): BF16 tensor-core forward,
    backward and Adam on the GPU; parameters as one packed FP32 vector."""

    def __init__(self, device: int = 0, stream=None):
        L = lib()
        self._L = L
        h = ctypes.c_void_p()
        rc = L.rbf_mlp_create(ctypes.byref(h), device, stream)
        if rc != RBF_OK:
            raise RbfError(rc, "rbf_mlp_create failed (no usable CUDA device?)")
        self._h = h
        self.n_params = int(L.rbf_mlp_num_params())
        self.out_scale = np.ones(4)

    def close(self):
        if getattr(self, "_h", None):
            self._L.rbf_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, rc):
        if rc != RBF_OK:
            raise RbfError(rc, self._L.rbf_mlp_last_error(self._h).decode())

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, np.float32)
        assert t.size == self.n_params
        self._ck(self._L.rbf_mlp_set_params(self._h, _ptr(t)))

    def get_params(self):
        out = np.empty(self.n_params, np.float32)
        self._ck(self._L.rbf_mlp_get_params(self._h, _ptr(out)))
        return out

    def set_data(self, xyz, radius, sdf, target):
        x = np.ascontiguousarray(xyz, np.float64)
        r = np.ascontiguousarray(radius, np.float32)
        s = np.ascontiguousarray(sdf, np.float32)
        t = np.ascontiguousarray(target, np.float32)
        self._keep = (x, r, s, t)
        self._ck(self._L.rbf_mlp_set_data(self._h, len(x), _ptr(x), _ptr(r), _ptr(s), _ptr(t)))

    def train(self, steps: int, batch: int, lr: float, seed: int):
        hist = np.zeros(max(steps, 1), np.float32)
        self._ck(self._L.rbf_mlp_train(self._h, int(steps), int(batch), float(lr), int(seed), _ptr(hist)))
        return hist[:steps]

    def gradient(self, sample_idx):
        idx = np.ascontiguousarray(sample_idx, np.int64)
        g = np.empty(self.n_params, np.float32)
        loss = ctypes.c_double()
        self._ck(self._L.rbf_mlp_gradient(self._h, len(idx), _ptr(idx), _ptr(g), ctypes.byref(loss)))
        return g, loss.value

    def predict(self, xyz, radius, sdf):
        x = np.ascontiguousarray(xyz, np.float64)
        r = np.ascontiguousarray(np.broadcast_to(radius, (len(x),)), np.float32)
        s = np.ascontiguousarray(sdf, np.float32)
        out = np.empty((len(x), 4), np.float32)
        self._ck(self._L.rbf_mlp_predict(self._h, len(x), _ptr(x), _ptr(r), _ptr(s), _ptr(out)))
        return out

    def warm_start(self, solver: "Solver", scale=1.0):
        """Write the prediction into the solver's fields: output c times
        scale * out_scale[c] (out_scale: the per-output factor the targets were
        divided by for training, ones by default)."""
        sc = np.ascontiguousarray(np.broadcast_to(np.asarray(scale, np.float64), (4,)) * self.out_scale, np.float64)
        self._ck(self._L.rbf_mlp_warm_start(self._h, solver._h, _ptr(sc)))

    def set_fused(self, fused: bool = True):
        """Training-step schedule: fused forward/backward kernels (default) or one
        GEMM launch per layer and pass."""
        self._ck(self._L.rbf_mlp_set_fused(self._h, int(bool(fused))))

    def launch_count(self) -> int:
        return int(self._L.rbf_mlp_launch_count(self._h))
