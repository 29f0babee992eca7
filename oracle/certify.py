"""Error certificates of computed FIDS levels (test infrastructure only,
like the rest of oracle/: only tests and the benchmark's CPU baseline use it).

A level of Eq. (3.16gu) reads M u = b with M = ahat I + K A (ahat =
b_m^{(m)} / Gamma(1 - gamma), K = diag(kappa^m)).  By Theorem 3.1 the
diagonal-dominance excess of M is at least ahat, so by Lemma 3.3
||M^{-1} y||_inf <= ||y||_inf / ahat for every y.

For a computed level u with defect d = b - M u, the exact level solution is
u + e with M e = d.  Lemma 3.3 alone gives ||e|| <= ||d|| / ahat; that bound
is attained only by defects that look like the operator's smoothest modes,
and at large n it cannot go below eps ||M||_inf / ahat ~ 1e-8 for ANY
double-precision u.  The certificate here sharpens it without losing rigour:
an approximate solution e~ of M e = d (any method: below, CG with a Strang
circulant preconditioner on numpy FFTs, a few digits suffice) and the defect
d2 = d - M e~ of the correction equation give

    ||u_exact - u||_inf <= ||e~||_inf + ||d2||_inf / ahat + (rounding terms),

both defects evaluated in double-double arithmetic (oracle.level_defect)
and the rounding terms bounded from sums of absolute values.
"""
from __future__ import annotations

import numpy as np

from . import level_defect

_U2 = 2.0 ** -104  # unit roundoff of the double-double accumulation


def _embed(t: np.ndarray) -> tuple[np.ndarray, int]:
    n = len(t)
    L = 1
    while L < 2 * n - 1:
        L *= 2
    col = np.zeros(L)
    col[:n] = t
    col[L - n + 1:] = t[1:][::-1]
    return np.fft.rfft(col), L


def _toeplitz_fft(spec: np.ndarray, L: int, v: np.ndarray) -> np.ndarray:
    """A v for the symmetric Toeplitz A whose even embedding has spectrum spec."""
    n = len(v)
    return np.fft.irfft(spec * np.fft.rfft(v, L), L)[:n]


def correction_solve(t, a, kappa, d, tol=1e-10, max_it=2000):
    """An approximate solution of (a I + K A) e = d: CG on the equivalent SPD
    system (a K^{-1} + A) e = K^{-1} d (A SPD by the proposition after
    Eq. (3.16x)) preconditioned by the Strang circulant a/kbar I + s(A) of
    Sec. 4.1, every product by numpy FFTs in FP64.  Its accuracy is not
    trusted: the certificate measures it through the defect of e."""
    t = np.asarray(t, dtype=np.float64)
    kappa = np.asarray(kappa, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    n = len(d)
    spec, L = _embed(t)
    cS = np.where(np.arange(n) <= n // 2, t, t[(n - np.arange(n)) % n])
    lam = np.fft.fft(cS).real
    pdiag = a / np.mean(kappa) + lam
    hinv = 1.0 / kappa
    S = lambda v: a * hinv * v + _toeplitz_fft(spec, L, v)
    Pinv = lambda r: np.fft.ifft(np.fft.fft(r) / pdiag).real
    rhs = hinv * d
    x = np.zeros(n)
    r = rhs.copy()
    nb = np.linalg.norm(rhs)
    if nb == 0.0:
        return x
    z = Pinv(r)
    p = z.copy()
    rz = r @ z
    for _ in range(max_it):
        q = S(p)
        al = rz / (p @ q)
        x += al * p
        r -= al * q
        if np.linalg.norm(r) <= tol * nb:
            break
        z = Pinv(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x


def _abs_terms(t, a, kappa, v, b):
    """Componentwise sum of absolute values of the terms of b - (a v + K A v):
    |b| + a|v| + kappa |A| |v| (|A| by an FFT product of nonnegative data, so
    accurate to a few ulps; doubled below for the bound)."""
    spec, L = _embed(np.abs(t))
    return np.abs(b) + a * np.abs(v) + kappa * np.maximum(_toeplitz_fft(spec, L, np.abs(v)), 0.0)


def certify_level(t, a, kappa, u, b):
    """Certified bound on ||u_exact - u||_inf for the level M u = b (a = ahat).
    Returns (bound, lemma33_bound), the second being ||d||_inf / a alone."""
    t = np.asarray(t, dtype=np.float64)
    kappa = np.asarray(kappa, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = len(u)
    d = level_defect(t, a, kappa, u, b)
    e = correction_solve(t, a, kappa, d)
    d2 = level_defect(t, a, kappa, e, d)
    # rounding of the two double-double evaluations: n terms per row, each
    # accumulation step off by at most a few 2^-104 of the running sums
    g = 4.0 * (n + 4) * _U2
    r1 = g * 2.0 * np.max(_abs_terms(t, a, kappa, u, b))
    r2 = g * 2.0 * np.max(_abs_terms(t, a, kappa, e, d))
    bound = np.max(np.abs(e)) + (np.max(np.abs(d2)) + r1 + r2) / a
    return float(bound), float(np.max(np.abs(d)) / a)
