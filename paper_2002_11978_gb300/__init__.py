"""Python binding of libtsfde (include/tsfde.h): the GB300 implementation of
the fast implicit difference scheme for the time-space fractional diffusion
equation with the integral fractional Laplacian (arXiv 2002.11978).

This module only marshals arguments: every step of the solver runs in the
CUDA library.  PyTorch provides device memory and the stream.  There is no
CPU fallback -- without the compiled library or a CUDA device the calls
raise.

Low-level names mirror the C ABI (``tsfde_setup``, ``tsfde_step``, ...);
``Solver`` wraps a context for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libtsfde.so")

TSFDE_OK, TSFDE_EINVAL, TSFDE_ENOMEM, TSFDE_ECUDA, TSFDE_ENOCONV = 0, 1, 2, 3, 4
TSFDE_EBREAKDOWN, TSFDE_ETIMEOUT, TSFDE_ESTATE, TSFDE_ENONFINITE, TSFDE_ENOTSUP = 5, 6, 7, 8, 9
TSFDE_FP64, TSFDE_MIXED, TSFDE_MIXED_DS = 0, 1, 2
TSFDE_STRANG, TSFDE_PRECOND_NONE = 0, 1
TSFDE_HISTORY_SOE, TSFDE_HISTORY_DIRECT = 0, 1
TSFDE_KRYLOV_BICGSTAB, TSFDE_KRYLOV_PCG, TSFDE_KRYLOV_AUTO = 0, 1, 2
TSFDE_ENGINE_AUTO, TSFDE_ENGINE_GRID, TSFDE_ENGINE_CLUSTER = 0, 1, 2

_dp = ctypes.POINTER(ctypes.c_double)


class tsfde_opts(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("kappa_mu", ctypes.c_int),
                ("krylov_tol", ctypes.c_double), ("max_it", ctypes.c_int),
                ("precision", ctypes.c_int), ("precond", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("inner_max_it", ctypes.c_int),
                ("soe_E", ctypes.c_int), ("soe_s", _dp), ("soe_w", _dp), ("profile", ctypes.c_int),
                ("barrier_timeout_cycles", ctypes.c_longlong), ("stream", ctypes.c_void_p),
                ("engine", ctypes.c_int), ("cluster_size", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("history", ctypes.c_int), ("krylov", ctypes.c_int),
                ("ckpt_stride", ctypes.c_int)]


class tsfde_step_info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("status", ctypes.c_int), ("iterations", ctypes.c_int),
                ("outer", ctypes.c_int), ("E_active", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("krylov", ctypes.c_int)]


class tsfde_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("failed_level", ctypes.c_int64),
                ("levels", ctypes.c_int64), ("iterations", ctypes.c_int64),
                ("min_iterations", ctypes.c_int), ("max_iterations", ctypes.c_int),
                ("outer", ctypes.c_int64), ("max_rel_residual", ctypes.c_double),
                ("E", ctypes.c_int), ("E_active_sum", ctypes.c_int64),
                ("pcg_levels", ctypes.c_int64)]


class tsfde_adjoint_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("failed_level", ctypes.c_int64),
                ("iterations", ctypes.c_int64), ("max_iterations", ctypes.c_int),
                ("max_rel_residual", ctypes.c_double), ("recomputed_levels", ctypes.c_int64)]


class tsfde_instance(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("gamma", ctypes.c_double), ("l", ctypes.c_double),
                ("T", ctypes.c_double), ("r", ctypes.c_double), ("n", ctypes.c_int64),
                ("soe_tol", ctypes.c_double), ("phi", ctypes.c_void_p), ("kappa", ctypes.c_void_p),
                ("f", ctypes.c_void_p)]


class tsfde_batch_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("failed_instance", ctypes.c_int),
                ("levels", ctypes.c_int64), ("iterations", ctypes.c_int64),
                ("outer", ctypes.c_int64), ("fp64_levels", ctypes.c_int64),
                ("max_rel_residual", ctypes.c_double)]


class tsfde_batch_plan(ctypes.Structure):
    _fields_ = [("classes", ctypes.c_int), ("split_n", ctypes.c_int64),
                ("cluster_size", ctypes.c_int * 2), ("clusters", ctypes.c_int * 2),
                ("probe_ms", ctypes.c_double)]


def plan_dict(p):
    return {"classes": p.classes, "split_n": p.split_n, "cluster_size": list(p.cluster_size),
            "clusters": list(p.clusters), "probe_ms": p.probe_ms}


class tsfde_timing(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int64), ("rhs_ms", ctypes.c_double),
                ("level_ms", ctypes.c_double)]


# (name, restype, argtypes) of every entry point in include/tsfde.h
_V = ctypes.c_void_p
_SIGNATURES = [
    ("tsfde_default_opts", ctypes.c_int, [ctypes.POINTER(tsfde_opts)]),
    ("tsfde_setup", ctypes.c_int, [ctypes.POINTER(_V), ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                   ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(tsfde_opts)]),
    ("tsfde_destroy", None, [_V]),
    ("tsfde_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("tsfde_last_error", ctypes.c_char_p, [_V]),
    ("tsfde_set_problem", ctypes.c_int, [_V, _V, _V, _V, _dp, ctypes.c_int,
                                         ctypes.POINTER(_V), _dp]),
    ("tsfde_reset", ctypes.c_int, [_V]),
    ("tsfde_step", ctypes.c_int, [_V, _V, _V, _V, _V, ctypes.POINTER(tsfde_step_info)]),
    ("tsfde_solve", ctypes.c_int, [_V, _V, _V, ctypes.POINTER(tsfde_solve_info)]),
    ("tsfde_get_soe", ctypes.c_int, [_V, ctypes.POINTER(ctypes.c_int), _dp, _dp]),
    ("tsfde_get_times", ctypes.c_int, [_V, _dp]),
    ("tsfde_get_symbol", ctypes.c_int, [_V, _dp]),
    ("tsfde_get_timing", ctypes.c_int, [_V, ctypes.POINTER(tsfde_timing)]),
    ("tsfde_get_engine", ctypes.c_int, [_V]),
    ("tsfde_adjoint", ctypes.c_int, [_V, _V, _V, _V, _V, ctypes.POINTER(tsfde_adjoint_info)]),
    ("tsfde_batch_setup", ctypes.c_int, [ctypes.POINTER(_V), ctypes.c_int,
                                         ctypes.POINTER(tsfde_instance), ctypes.c_int64,
                                         ctypes.POINTER(tsfde_opts)]),
    ("tsfde_batch_solve", ctypes.c_int, [_V, ctypes.c_int64, ctypes.POINTER(_V),
                                         ctypes.POINTER(tsfde_batch_info)]),
    ("tsfde_batch_instance_stats", ctypes.c_int, [_V, ctypes.c_int, ctypes.POINTER(tsfde_step_info)]),
    ("tsfde_batch_shape", ctypes.c_int, [_V, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    ("tsfde_batch_destroy", None, [_V]),
    ("tsfde_batch_setup_plan", ctypes.c_int, [ctypes.POINTER(_V), ctypes.c_int,
                                              ctypes.POINTER(tsfde_instance), ctypes.c_int64,
                                              ctypes.POINTER(tsfde_opts), ctypes.POINTER(tsfde_batch_plan)]),
    ("tsfde_batch_get_plan", ctypes.c_int, [_V, ctypes.POINTER(tsfde_batch_plan)]),
    ("tsfde_batch_tune", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(tsfde_instance), ctypes.c_int64,
                                        ctypes.POINTER(tsfde_opts), ctypes.c_int64,
                                        ctypes.POINTER(tsfde_batch_plan), ctypes.POINTER(tsfde_batch_plan),
                                        ctypes.POINTER(ctypes.c_int)]),
    ("tsfde_get_level_stats", ctypes.c_int, [_V, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.POINTER(tsfde_step_info)]),
    ("tsfde_get_solution", ctypes.c_int, [_V, _V]),
    ("tsfde_toeplitz_apply", ctypes.c_int, [_V, _V, _V, ctypes.c_int]),
    ("tsfde_operator_apply", ctypes.c_int, [_V, ctypes.c_double, _V, _V, _V, ctypes.c_int]),
    ("tsfde_precond_apply", ctypes.c_int, [_V, ctypes.c_double, ctypes.c_double, _V, _V,
                                           ctypes.c_int]),
    ("tsfde_linear_solve", ctypes.c_int, [_V, ctypes.c_double, _V, _V, _V,
                                          ctypes.POINTER(tsfde_step_info)]),
    ("tsfde_toeplitz_apply_static", ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                   ctypes.c_double, ctypes.c_int64, _V, _V, _V]),
    ("tsfde_probe_l2_read", ctypes.c_int, [_V, ctypes.c_size_t, ctypes.c_int, _V]),
]

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtsfde.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} not found: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        for name, res, args in _SIGNATURES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def exported_names():
    return [s[0] for s in _SIGNATURES]


class TsfdeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _check(status: int, ctx=None):
    if status != TSFDE_OK:
        lib = load_library()
        detail = lib.tsfde_last_error(ctx).decode() if ctx else ""
        raise TsfdeError(status, f"{lib.tsfde_strerror(status).decode()}: {detail}")


def _dev(t, n=None, name="tensor"):
    """Device pointer of a contiguous CUDA float64 tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, has {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def default_opts() -> tsfde_opts:
    o = tsfde_opts()
    _check(load_library().tsfde_default_opts(ctypes.byref(o)))
    return o


class Solver:
    """One FIDS problem: tsfde_setup + tsfde_set_problem + stepping."""

    def __init__(self, alpha, gamma, l, T, n, M, r, soe_tol=1e-12, *, precision="fp64",
                 precond="strang", krylov_tol=1e-12, max_it=2000, inner_tol=1e-2,
                 max_outer=60, inner_max_it=40, mu=None, kappa_mu=None, soe=None, barrier_timeout_cycles=0,
                 profile=False, stream=None, engine="auto", warm_start=False, history="soe",
                 krylov="bicgstab", ckpt_stride=0):
        lib = load_library()
        o = default_opts()
        o.krylov = {"bicgstab": TSFDE_KRYLOV_BICGSTAB, "pcg": TSFDE_KRYLOV_PCG,
                    "auto": TSFDE_KRYLOV_AUTO}[krylov]
        o.history = {"soe": TSFDE_HISTORY_SOE, "direct": TSFDE_HISTORY_DIRECT}[history]
        o.warm_start = _warm(warm_start)
        o.ckpt_stride = int(ckpt_stride)
        o.engine = {"auto": TSFDE_ENGINE_AUTO, "grid": TSFDE_ENGINE_GRID,
                    "cluster": TSFDE_ENGINE_CLUSTER}[engine]
        o.krylov_tol = krylov_tol
        o.max_it = max_it
        o.precision = {"fp64": TSFDE_FP64, "mixed": TSFDE_MIXED, "mixed_ds": TSFDE_MIXED_DS}[precision]
        o.precond = {"strang": TSFDE_STRANG, "none": TSFDE_PRECOND_NONE}[precond]
        o.inner_tol = inner_tol
        o.max_outer = max_outer
        o.inner_max_it = inner_max_it
        o.mu = 0.0 if mu is None else mu
        o.kappa_mu = 0 if kappa_mu is None else kappa_mu
        o.barrier_timeout_cycles = barrier_timeout_cycles
        o.profile = 1 if profile else 0
        self._keep = []
        if soe is not None:
            s = np.ascontiguousarray(soe[0], dtype=np.float64)
            w = np.ascontiguousarray(soe[1], dtype=np.float64)
            self._keep += [s, w]
            o.soe_E = len(s)
            o.soe_s = s.ctypes.data_as(_dp)
            o.soe_w = w.ctypes.data_as(_dp)
        self.stream = stream
        o.stream = _stream_handle(stream)
        self.n, self.M = int(n), int(M)
        self.m = 0  # current time level
        self.ckpt_stride = int(ckpt_stride)
        self.problem_token = None  # changes with every set_problem
        self.ctx = ctypes.c_void_p()
        _check(lib.tsfde_setup(ctypes.byref(self.ctx), alpha, gamma, l, T, self.n, self.M, r,
                               soe_tol, ctypes.byref(o)))
        self.lib = lib

    def close(self):
        if self.ctx:
            self.lib.tsfde_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- problem data
    def set_problem(self, phi, kappa0, kappa1=None, theta=None, F=(), G=None):
        n, M = self.n, self.M
        th = None
        if theta is not None:
            th = np.ascontiguousarray(theta, dtype=np.float64)
            assert th.shape == (M + 1,)
        F = list(F)
        rank = len(F)
        Farr = (ctypes.c_void_p * max(rank, 1))(*[_dev(f, n, "F").value for f in F])
        Garr = None
        if rank:
            Garr = np.ascontiguousarray(G, dtype=np.float64).reshape(rank, M + 1)
        self._problem_keep = [phi, kappa0, kappa1, F, th, Garr]
        _check(self.lib.tsfde_set_problem(
            self.ctx, _dev(phi, n, "phi"), _dev(kappa0, n, "kappa0"), _dev(kappa1, n, "kappa1"),
            None if th is None else th.ctypes.data_as(_dp), rank,
            ctypes.cast(Farr, ctypes.POINTER(ctypes.c_void_p)),
            None if Garr is None else Garr.ctypes.data_as(_dp)), self.ctx)
        self.m = 0
        self.problem_token = object()

    def set_problem_from(self, prob):
        """Feed a tsfde_inputs.Problem (separable form) through set_problem."""
        import torch
        dev = torch.device("cuda")
        t = self.times()
        to = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
        F = [to(f) for f in prob.F]
        self.set_problem(to(prob.phi), to(prob.kappa0),
                         None if prob.kappa1 is None else to(prob.kappa1),
                         prob.theta_values(t), F, prob.G_values(t) if F else None)

    def reset(self):
        _check(self.lib.tsfde_reset(self.ctx), self.ctx)
        self.m = 0

    # ---- stepping
    def step(self, kappa_m=None, f_m=None, u_out=None, rhs_out=None, sync=True):
        info = tsfde_step_info()
        rc = self.lib.tsfde_step(self.ctx, _dev(kappa_m, self.n, "kappa_m"),
                                 _dev(f_m, self.n, "f_m"), _dev(u_out, self.n, "u_out"),
                                 _dev(rhs_out, self.n, "rhs_out"),
                                 ctypes.byref(info) if sync else None)
        if rc == TSFDE_OK or (sync and info.m == self.m + 1):
            self.m += 1  # the level was computed even if its solve failed
        _check(rc, self.ctx)
        return _info_dict(info) if sync else None

    def solve(self, u_final, u_all=None, sync=True):
        info = tsfde_solve_info()
        _check(self.lib.tsfde_solve(self.ctx, _dev(u_final, self.n, "u_final"),
                                    _dev(u_all, (self.M + 1) * self.n, "u_all"),
                                    ctypes.byref(info) if sync else None), self.ctx)
        self.m = self.M
        return _info_dict(info) if sync else None

    # ---- tables
    def soe(self):
        E = ctypes.c_int(0)
        _check(self.lib.tsfde_get_soe(self.ctx, ctypes.byref(E), None, None), self.ctx)
        s = np.zeros(E.value)
        w = np.zeros(E.value)
        _check(self.lib.tsfde_get_soe(self.ctx, ctypes.byref(E), s.ctypes.data_as(_dp),
                                      w.ctypes.data_as(_dp)), self.ctx)
        return s, w

    def times(self):
        t = np.zeros(self.M + 1)
        _check(self.lib.tsfde_get_times(self.ctx, t.ctypes.data_as(_dp)), self.ctx)
        return t

    @property
    def engine(self) -> str:
        """'grid' or 'cluster': where the mixed level solves run their FP32 inner solves."""
        return {TSFDE_ENGINE_GRID: "grid", TSFDE_ENGINE_CLUSTER: "cluster"}[
            self.lib.tsfde_get_engine(self.ctx)]

    def timing(self):
        t = tsfde_timing()
        _check(self.lib.tsfde_get_timing(self.ctx, ctypes.byref(t)), self.ctx)
        return _info_dict(t)

    def level_stats(self, m0, m1):
        out = (tsfde_step_info * (m1 - m0 + 1))()
        _check(self.lib.tsfde_get_level_stats(self.ctx, m0, m1, out), self.ctx)
        return [_info_dict(x) for x in out]

    def current_solution(self, u):
        _check(self.lib.tsfde_get_solution(self.ctx, _dev(u, self.n, "u")), self.ctx)

    def symbol(self):
        t = np.zeros(self.n)
        _check(self.lib.tsfde_get_symbol(self.ctx, t.ctypes.data_as(_dp)), self.ctx)
        return t

    # ---- single operations
    def toeplitz_apply(self, v, y, precision="fp64"):
        _check(self.lib.tsfde_toeplitz_apply(self.ctx, _dev(v, self.n, "v"), _dev(y, self.n, "y"),
                                             _prec(precision)), self.ctx)

    def operator_apply(self, a, kappa, v, y, precision="fp64"):
        _check(self.lib.tsfde_operator_apply(self.ctx, a, _dev(kappa, self.n, "kappa"),
                                             _dev(v, self.n, "v"), _dev(y, self.n, "y"),
                                             _prec(precision)), self.ctx)

    def precond_apply(self, a, kbar, v, z, precision="fp64"):
        _check(self.lib.tsfde_precond_apply(self.ctx, a, kbar, _dev(v, self.n, "v"),
                                            _dev(z, self.n, "z"), _prec(precision)), self.ctx)

    def adjoint(self, u_all, dJ_duM, grad_kappa, grad_f):
        """Discrete adjoint of the FIDS march (tsfde_adjoint): given the forward
        levels u_all ((M+1) x n, as solve() writes them) and dJ/du^M, write
        dJ/dkappa and dJ/df for a time-independent kappa and f.  u_all = None
        recomputes the levels from the checkpoints of the last march (a
        solver made with ckpt_stride != 0)."""
        if u_all is not None and tuple(u_all.shape) != (self.M + 1, self.n):
            raise ValueError(f"u_all must be ({self.M + 1}, {self.n})")
        info = tsfde_adjoint_info()
        _check(self.lib.tsfde_adjoint(self.ctx, _dev(u_all, None, "u_all"),
                                      _dev(dJ_duM, self.n, "dJ_duM"),
                                      _dev(grad_kappa, self.n, "grad_kappa"),
                                      _dev(grad_f, self.n, "grad_f"), ctypes.byref(info)), self.ctx)
        return _info_dict(info)

    def linear_solve(self, a, kappa, b, x):
        info = tsfde_step_info()
        _check(self.lib.tsfde_linear_solve(self.ctx, a, _dev(kappa, self.n, "kappa"),
                                           _dev(b, self.n, "b"), _dev(x, self.n, "x"),
                                           ctypes.byref(info)), self.ctx)
        return _info_dict(info)


class BatchSolver:
    """Many independent FIDS problems over a common M (tsfde_batch_*).

    instances: list of dicts with alpha, gamma, n, phi, kappa, f (CUDA
    float64 tensors of n entries; kappa and f time independent) and optional
    l (1), T (1), r ((2-gamma)/gamma), soe_tol (1e-12)."""

    def __init__(self, instances, M, *, precision="mixed", precond="strang", krylov_tol=1e-12,
                 max_it=2000, inner_tol=1e-2, max_outer=60, inner_max_it=40, mu=None,
                 kappa_mu=None, stream=None, cluster_size=0, warm_start=False, plan=None,
                 krylov="bicgstab"):
        """plan: None (the default launch plan), a tsfde_batch_plan, or a dict
        as batch_tune / .plan return."""
        lib = load_library()
        o, arr = _batch_args(instances, precision, precond, krylov_tol, max_it, inner_tol, max_outer,
                             inner_max_it, mu, kappa_mu, stream, cluster_size, warm_start, krylov)
        self.ns = [int(d["n"]) for d in instances]
        self.lib = lib
        self.B, self.M = len(instances), int(M)
        self.ctx = ctypes.c_void_p()
        pp = None if plan is None else ctypes.byref(_as_plan(plan))
        _check(lib.tsfde_batch_setup_plan(ctypes.byref(self.ctx), self.B, arr, self.M, ctypes.byref(o), pp))

    @property
    def plan(self):
        p = tsfde_batch_plan()
        _check(self.lib.tsfde_batch_get_plan(self.ctx, ctypes.byref(p)))
        return plan_dict(p)

    def __del__(self):
        if getattr(self, "ctx", None):
            self.lib.tsfde_batch_destroy(self.ctx)
            self.ctx = None

    @property
    def shape(self):
        c, q = ctypes.c_int(), ctypes.c_int()
        _check(self.lib.tsfde_batch_shape(self.ctx, ctypes.byref(c), ctypes.byref(q)))
        return c.value, q.value

    def solve(self, u_final, levels=0):
        """u_final: list of B CUDA float64 tensors (n_i entries) receiving
        u^levels (levels = 0: u^M)."""
        if len(u_final) != self.B:
            raise ValueError("need one output per instance")
        ptrs = (ctypes.c_void_p * self.B)(*[_dev(u, n, "u_final").value for u, n in zip(u_final, self.ns)])
        info = tsfde_batch_info()
        rc = self.lib.tsfde_batch_solve(self.ctx, int(levels), ptrs, ctypes.byref(info))
        out = _info_dict(info)
        if rc != TSFDE_OK:
            raise TsfdeError(rc, f"{self.lib.tsfde_strerror(rc).decode()}: batch solve, {out}")
        return out

    def instance_stats(self, i):
        info = tsfde_step_info()
        _check(self.lib.tsfde_batch_instance_stats(self.ctx, i, ctypes.byref(info)))
        return _info_dict(info)


def _batch_args(instances, precision="mixed", precond="strang", krylov_tol=1e-12, max_it=2000,
                inner_tol=1e-2, max_outer=60, inner_max_it=40, mu=None, kappa_mu=None, stream=None,
                cluster_size=0, warm_start=False, krylov="bicgstab"):
    o = default_opts()
    o.krylov = {"bicgstab": TSFDE_KRYLOV_BICGSTAB, "pcg": TSFDE_KRYLOV_PCG, "auto": TSFDE_KRYLOV_AUTO}[krylov]
    o.cluster_size = cluster_size
    o.warm_start = _warm(warm_start)
    o.krylov_tol = krylov_tol
    o.max_it = max_it
    o.precision = {"fp64": TSFDE_FP64, "mixed": TSFDE_MIXED}[precision]
    o.precond = {"strang": TSFDE_STRANG, "none": TSFDE_PRECOND_NONE}[precond]
    o.inner_tol = inner_tol
    o.max_outer = max_outer
    o.inner_max_it = inner_max_it
    o.mu = 0.0 if mu is None else mu
    o.kappa_mu = 0 if kappa_mu is None else kappa_mu
    if stream is not None:
        o.stream = _stream_handle(stream)
    B = len(instances)
    arr = (tsfde_instance * B)()
    for i, d in enumerate(instances):
        g = float(d["gamma"])
        n = int(d["n"])
        arr[i] = tsfde_instance(float(d["alpha"]), g, float(d.get("l", 1.0)), float(d.get("T", 1.0)),
                                float(d.get("r", (2.0 - g) / g)), n, float(d.get("soe_tol", 1e-12)),
                                _dev(d["phi"], n, "phi"), _dev(d["kappa"], n, "kappa"),
                                _dev(d["f"], n, "f"))
    return o, arr


def _as_plan(p):
    if isinstance(p, tsfde_batch_plan):
        return p
    q = tsfde_batch_plan()
    q.classes = int(p["classes"])
    q.split_n = int(p.get("split_n", 0))
    for k in range(2):
        q.cluster_size[k] = int(p["cluster_size"][k])
    return q


def batch_tune(instances, M, probe_levels=4, **kw):
    """Autotune the batched launch plan (tsfde_batch_tune): returns
    (best plan, list of every timed plan) as dicts; kw as BatchSolver."""
    lib = load_library()
    o, arr = _batch_args(instances, **kw)
    best = tsfde_batch_plan()
    tried = (tsfde_batch_plan * 16)()
    nt = ctypes.c_int(16)
    _check(lib.tsfde_batch_tune(len(instances), arr, int(M), ctypes.byref(o), int(probe_levels),
                                ctypes.byref(best), tried, ctypes.byref(nt)))
    return plan_dict(best), [plan_dict(tried[k]) for k in range(nt.value)]


def toeplitz_apply_static(alpha, n, v, y, l=1.0, mu=None, kappa_mu=None, stream=None):
    """y = A v through tsfde_toeplitz_apply_static (no context, no device
    allocation; n <= 16383)."""
    lib = load_library()
    _check(lib.tsfde_toeplitz_apply_static(alpha, 0.0 if mu is None else mu,
                                           0 if kappa_mu is None else kappa_mu, l, int(n),
                                           _dev(v, n, "v"), _dev(y, n, "y"),
                                           _stream_handle(stream)))


def probe_l2_read(buf, reps, stream=None):
    """Enqueue tsfde_probe_l2_read over the CUDA tensor buf (its whole
    storage, 16-byte aligned) `reps` times on `stream`; time it with events
    on that stream."""
    lib = load_library()
    nbytes = buf.numel() * buf.element_size()
    if not buf.is_cuda or not buf.is_contiguous():
        raise ValueError("buf must be a contiguous CUDA tensor")
    _check(lib.tsfde_probe_l2_read(ctypes.c_void_p(buf.data_ptr()), nbytes, int(reps),
                                   _stream_handle(stream)))


def _warm(w):
    """warm_start option: False/0 (x0 = 0), True/1 (u^{m-1}) or
    "extrapolate"/2 (cubic extrapolation in the level index from
    u^{m-4} .. u^{m-1})."""
    if w in ("extrapolate", 2):
        return 2
    return 1 if w else 0


def _prec(p):
    return {"fp64": TSFDE_FP64, "mixed": TSFDE_MIXED, "fp32": TSFDE_MIXED,
            "mixed_ds": TSFDE_MIXED_DS, "ds": TSFDE_MIXED_DS}[p]


def _info_dict(info):
    return {f: getattr(info, f) for f, _ in info._fields_}
