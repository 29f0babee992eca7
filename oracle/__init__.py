"""CPU oracle for FIDS/DIDS (arXiv 2002.11978) -- TEST INFRASTRUCTURE ONLY.

A thin ctypes wrapper over ``oracle.c`` (plain C, IEEE double, dense LU and
direct O(M^2 n) history sums).  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares
no code with the CUDA path and never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it (gcc, no fast-math, no
    FMA contraction so x86 and Arm give the same bits)."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC),
                                          os.path.getmtime(os.path.join(_HERE, "oracle.h")))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-fopenmp",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        L.or_c1alpha.restype = ctypes.c_double
        L.or_c1alpha.argtypes = [ctypes.c_double]
        L.or_ifl_symbol.restype = ctypes.c_int
        L.or_ifl_symbol.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int64, ctypes.c_double, _dp]
        L.or_graded_mesh.restype = ctypes.c_int
        L.or_graded_mesh.argtypes = [ctypes.c_double, ctypes.c_int64, ctypes.c_double, _dp, _dp]
        L.or_mesh_gap.restype = ctypes.c_double
        L.or_mesh_gap.argtypes = [ctypes.c_double, ctypes.c_int64, ctypes.c_double,
                                  ctypes.c_int64, ctypes.c_int64]
        L.or_l1_weight.restype = ctypes.c_double
        L.or_l1_weight.argtypes = [ctypes.c_double, ctypes.c_int64, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int64, ctypes.c_int64]
        L.or_soe_build.restype = ctypes.c_int
        L.or_soe_build.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, _dp, _dp]
        L.or_soe_rel_err.restype = ctypes.c_double
        L.or_soe_rel_err.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, _dp, _dp, ctypes.c_int]
        L.or_fids_weight.restype = ctypes.c_double
        L.or_fids_weight.argtypes = [ctypes.c_double, ctypes.c_int64, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_int, _dp, _dp]
        L.or_lu_solve.restype = ctypes.c_int
        L.or_lu_solve.argtypes = [ctypes.c_int64, _dp, _dp]
        L.or_level_rhs.restype = ctypes.c_int
        L.or_level_rhs.argtypes = [ctypes.POINTER(OrProblem), ctypes.c_int, ctypes.c_int64, _dp, _dp, _dp]
        L.or_level_defect.restype = None
        L.or_level_defect.argtypes = [ctypes.c_int64, _dp, ctypes.c_double, _dp, _dp, _dp, _dp]
        L.or_set_threads.restype = None
        L.or_set_threads.argtypes = [ctypes.c_int]
        L.or_get_threads.restype = ctypes.c_int
        L.or_get_threads.argtypes = []
        L.or_toeplitz_matvec.restype = None
        L.or_toeplitz_matvec.argtypes = [ctypes.c_int64, _dp, _dp, _dp]
        L.or_strang_column.restype = None
        L.or_strang_column.argtypes = [ctypes.c_int64, _dp, _dp]
        L.or_strang_eigs.restype = None
        L.or_strang_eigs.argtypes = [ctypes.c_int64, _dp, _dp]
        L.or_march.restype = ctypes.c_int
        L.or_march.argtypes = [ctypes.POINTER(OrProblem), ctypes.c_int, _dp]
        L.or_adjoint.restype = ctypes.c_int
        L.or_adjoint.argtypes = [ctypes.POINTER(OrProblem), _dp, _dp, _dp, _dp]
        _lib = L
    return _lib


class OrProblem(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("gamma", ctypes.c_double),
                ("l", ctypes.c_double), ("T", ctypes.c_double), ("r", ctypes.c_double),
                ("mu", ctypes.c_double), ("kappa_mu", ctypes.c_int),
                ("n", ctypes.c_int64), ("M", ctypes.c_int64),
                ("phi", _dp), ("kappa", _dp), ("f", _dp),
                ("soe_E", ctypes.c_int), ("soe_s", _dp), ("soe_w", _dp),
                ("levels", ctypes.c_int64)]


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def c1alpha(alpha: float) -> float:
    """c_{1,alpha}, Eq. (1.4)."""
    return lib().or_c1alpha(alpha)


def default_mu(alpha: float) -> tuple[float, int]:
    """The paper's main splitting choice mu = 1 + alpha/2, kappa_mu = 1
    (Sec. 2, Eq. (2.11); Tables 1-4, 7-11)."""
    return 1.0 + 0.5 * alpha, 1


def ifl_symbol(alpha: float, n: int, l: float = 1.0, mu: float | None = None,
               kappa_mu: int | None = None) -> np.ndarray:
    """First column of A, Eq. (3.16x)."""
    if mu is None:
        mu, km = default_mu(alpha)
        kappa_mu = km if kappa_mu is None else kappa_mu
    if kappa_mu is None:
        kappa_mu = 2 if mu == 2.0 else 1
    t = np.zeros(n)
    rc = lib().or_ifl_symbol(alpha, mu, kappa_mu, n, l, _ptr(t))
    if rc != 0:
        raise ValueError("bad IFL parameters")
    return t


def dense_A(t: np.ndarray) -> np.ndarray:
    n = len(t)
    idx = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :])
    return t[idx]


def graded_mesh(T: float, M: int, r: float):
    t = np.zeros(M + 1)
    tau = np.zeros(M + 1)
    if lib().or_graded_mesh(T, M, r, _ptr(t), _ptr(tau)) != 0:
        raise ValueError("bad mesh parameters")
    return t, tau


def l1_weight(T, M, r, gamma, m, k) -> float:
    """a_k^{(m)}, Eq. (2.8)."""
    return lib().or_l1_weight(T, M, r, gamma, m, k)


def soe_build(gamma: float, delta: float, T: float, tol: float, maxE: int = 4000):
    """Plain trapezoid SOE table (Lemma 2.2), verified to relative tol."""
    s = np.zeros(maxE)
    w = np.zeros(maxE)
    E = lib().or_soe_build(gamma, delta, T, tol, maxE, _ptr(s), _ptr(w))
    if E < 0:
        raise RuntimeError("SOE construction failed")
    return s[:E].copy(), w[:E].copy()


def soe_rel_err(gamma, delta, T, s, w, nsamp: int = 20001) -> float:
    s = _f64(s)
    w = _f64(w)
    return lib().or_soe_rel_err(gamma, delta, T, len(s), _ptr(s), _ptr(w), nsamp)


def fids_weight(T, M, r, gamma, m, k, s, w) -> float:
    """b_k^{(m)} (definition under Eq. (lem2.3))."""
    s = _f64(s)
    w = _f64(w)
    return lib().or_fids_weight(T, M, r, gamma, m, k, len(s), _ptr(s), _ptr(w))


def set_threads(t: int) -> None:
    """Threads of the LU row updates (default 1; the result does not change)."""
    lib().or_set_threads(int(t))


def get_threads() -> int:
    return int(lib().or_get_threads())


def lu_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    A = _f64(A).copy()
    x = _f64(b).copy()
    if lib().or_lu_solve(len(x), _ptr(A), _ptr(x)) != 0:
        raise np.linalg.LinAlgError("zero pivot")
    return x


def toeplitz_matvec(t: np.ndarray, v: np.ndarray) -> np.ndarray:
    t = _f64(t)
    v = _f64(v)
    y = np.zeros_like(v)
    lib().or_toeplitz_matvec(len(v), _ptr(t), _ptr(v), _ptr(y))
    return y


def strang_column(t: np.ndarray) -> np.ndarray:
    t = _f64(t)
    c = np.zeros_like(t)
    lib().or_strang_column(len(t), _ptr(t), _ptr(c))
    return c


def strang_eigs(t: np.ndarray) -> np.ndarray:
    t = _f64(t)
    lam = np.zeros_like(t)
    lib().or_strang_eigs(len(t), _ptr(t), _ptr(lam))
    return lam


def _problem(alpha, gamma, l, T, r, n, M, phi, kappa, f, mu=None, kappa_mu=None,
             soe=None, levels=0):
    if mu is None:
        mu, km = default_mu(alpha)
        kappa_mu = km if kappa_mu is None else kappa_mu
    if kappa_mu is None:
        kappa_mu = 2 if mu == 2.0 else 1
    keep = [_f64(phi), _f64(kappa), _f64(f)]
    assert keep[0].shape == (n,)
    assert keep[1].shape == (M + 1, n) and keep[2].shape == (M + 1, n)
    if soe is not None:
        keep += [_f64(soe[0]), _f64(soe[1])]
    p = OrProblem(alpha, gamma, l, T, r, mu, kappa_mu, n, M,
                  _ptr(keep[0]), _ptr(keep[1]), _ptr(keep[2]),
                  0 if soe is None else len(keep[3]),
                  None if soe is None else _ptr(keep[3]),
                  None if soe is None else _ptr(keep[4]), levels)
    return p, keep


def march(scheme: str, alpha, gamma, l, T, r, n, M, phi, kappa, f, mu=None,
          kappa_mu=None, soe=None, levels: int = 0) -> np.ndarray:
    """Time march with dense LU per level.  scheme = 'DIDS' (Eq. (3.16))
    or 'FIDS' (Eq. (3.15), needs soe=(s, w)).  kappa, f: (M+1, n) tables.
    Returns U of shape (M+1, n); with levels > 0 only rows 0..levels are
    computed (the rest stay zero)."""
    p, keep = _problem(alpha, gamma, l, T, r, n, M, phi, kappa, f, mu, kappa_mu, soe, levels)
    if scheme == "FIDS" and soe is None:
        raise ValueError("FIDS needs an SOE table")
    U = np.zeros((M + 1, n))
    rc = lib().or_march(ctypes.byref(p), 0 if scheme == "DIDS" else 1, _ptr(U))
    if rc != 0:
        raise RuntimeError(f"or_march failed ({rc})")
    return U


def level_rhs(scheme: str, alpha, gamma, l, T, r, n, M, m, U, f_m, soe=None, mu=None,
              kappa_mu=None) -> np.ndarray:
    """Right-hand side b^m of level m of Eq. (3.16gu) (FIDS, needs soe) or
    Eq. (4.1) (DIDS) from the levels U (rows 0..m-1, e.g. a GPU march) and
    the source f^m: the direct history sums with the direct weights."""
    if mu is None:
        mu, km = default_mu(alpha)
        kappa_mu = km if kappa_mu is None else kappa_mu
    if kappa_mu is None:
        kappa_mu = 2 if mu == 2.0 else 1
    Uc = np.ascontiguousarray(U[:m], dtype=np.float64)
    assert Uc.shape == (m, n)
    fm = _f64(f_m)
    keep = [Uc, fm]
    if soe is not None:
        keep += [_f64(soe[0]), _f64(soe[1])]
    p = OrProblem(alpha, gamma, l, T, r, mu, kappa_mu, n, M, _ptr(Uc), None, None,
                  0 if soe is None else len(keep[2]), None if soe is None else _ptr(keep[2]),
                  None if soe is None else _ptr(keep[3]), 0)
    rhs = np.zeros(n)
    if lib().or_level_rhs(ctypes.byref(p), 0 if scheme == "DIDS" else 1, m, _ptr(Uc), _ptr(fm), _ptr(rhs)) != 0:
        raise ValueError("bad level or missing SOE table")
    return rhs


def level_defect(t, a, kappa, u, b) -> np.ndarray:
    """d = b - (a u + kappa .* (A u)) with A the symmetric Toeplitz matrix of
    first column t, in double-double arithmetic rounded once."""
    t, kappa, u, b = _f64(t), _f64(kappa), _f64(u), _f64(b)
    d = np.zeros(len(u))
    lib().or_level_defect(len(u), _ptr(t), float(a), _ptr(kappa), _ptr(u), _ptr(b), _ptr(d))
    return d


def adjoint(alpha, gamma, l, T, r, n, M, phi, kappa_x, f_x, u_obs, soe, mu=None,
            kappa_mu=None):
    """Dense adjoint of the FIDS march for J = 1/2||u^M - u_obs||^2 with
    time-independent kappa(x) and f(x).  Returns (J, U, dJ/dkappa, dJ/df)."""
    kap = np.tile(_f64(kappa_x), (M + 1, 1))
    ff = np.tile(_f64(f_x), (M + 1, 1))
    U = march("FIDS", alpha, gamma, l, T, r, n, M, phi, kap, ff, mu, kappa_mu, soe)
    p, keep = _problem(alpha, gamma, l, T, r, n, M, phi, kap, ff, mu, kappa_mu, soe)
    gk = np.zeros(n)
    gf = np.zeros(n)
    uo = _f64(u_obs)
    rc = lib().or_adjoint(ctypes.byref(p), _ptr(U), _ptr(uo), _ptr(gk), _ptr(gf))
    if rc != 0:
        raise RuntimeError("or_adjoint failed")
    J = 0.5 * float(np.sum((U[M] - uo) ** 2))
    return J, U, gk, gf


def errors(U: np.ndarray, Uex: np.ndarray, h: float):
    """Err_inf = max_j ||E^j||_inf and Err_2 = max_j ||E^j||_2 with the
    discrete norm ||v||_2 = sqrt(h sum v_i^2) (Sec. 5)."""
    E = U - Uex
    return float(np.max(np.abs(E))), float(np.max(np.sqrt(h * np.sum(E * E, axis=1))))
