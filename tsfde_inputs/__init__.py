"""Seeded synthetic inputs for the time-space fractional diffusion problem
(Eq. (1.1) of arXiv 2002.11978).

This module defines PROBLEM DATA only -- the initial value phi, the
diffusivity kappa(x, t), the source f(x, t) and, where known, the exact
solution -- evaluated at caller-supplied points.  It holds none of the
scheme's arithmetic (no mesh weights, no symbol, no solver) and is the one
module that both the CPU oracle and the CUDA path consume.

Separable forms are exposed as factors so the CUDA path can take them through
its C ABI:
    kappa(x_i, t) = kappa0_i + theta(t) * kappa1_i
    f(x_i, t)     = sum_r G_r(t) * F_r[i]
Non-separable problems (Example 2) provide callables instead.

Random fields use numpy's PCG64 with the stated seeds.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np


def interior_nodes(n: int, l: float = 1.0) -> np.ndarray:
    """x_i = -l + i h, h = 2l/(n+1), i = 1..n: the n interior grid points of
    Omega = (-l, l) (Sec. 3.1 with paper N = n + 1 intervals)."""
    h = 2.0 * l / (n + 1)
    return -l + h * np.arange(1, n + 1, dtype=np.float64)


def terminating_2f1(a: float, s: int, z: np.ndarray) -> np.ndarray:
    """2F1(a, -s; 1/2; z) for integer s >= 0: a polynomial of degree s in z."""
    z = np.asarray(z, dtype=np.float64)
    tot = np.zeros_like(z)
    coef = 1.0
    for k in range(s + 1):
        tot = tot + coef * z ** k
        coef *= (a + k) * (-s + k) / ((0.5 + k) * (k + 1))
    return tot


def frac_lap_bump_constant(alpha: float, s: int) -> float:
    """2^a Gamma((a+1)/2) Gamma(s+1+a/2) / (sqrt(pi) Gamma(s+1)): the factor in
    (-Delta)^{a/2} (1-x^2)_+^{s+a/2} = const * 2F1((a+1)/2, -s; 1/2; x^2)
    (Example 1, Sec. 5)."""
    return (2.0 ** alpha * math.gamma(0.5 * (alpha + 1.0)) * math.gamma(s + 1.0 + 0.5 * alpha)
            / (math.sqrt(math.pi) * math.gamma(s + 1.0)))


def frac_lap_bump(alpha: float, s: int, x: np.ndarray) -> np.ndarray:
    """Exact (-Delta)^{a/2} (1-x^2)_+^{s+a/2} for |x| < 1."""
    return frac_lap_bump_constant(alpha, s) * terminating_2f1(0.5 * (alpha + 1.0), s, x * x)


def fourier_field(n: int, seed: int, l: float = 1.0, modes: int = 16) -> np.ndarray:
    """F(x) = sum_{k=1}^{16} (a_k cos(k pi x / l) + b_k sin(k pi x / l)) / k^2,
    a_k, b_k ~ N(0, 1) (PCG64(seed)), on the interior nodes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.standard_normal(modes)
    b = rng.standard_normal(modes)
    x = interior_nodes(n, l)
    F = np.zeros(n)
    for k in range(1, modes + 1):
        F += (a[k - 1] * np.cos(k * math.pi * x / l) + b[k - 1] * np.sin(k * math.pi * x / l)) / k ** 2
    return F


def gaussian_field(n: int, seed: int, l: float = 1.0, corr: float = 0.1,
                   var: float = 0.5) -> np.ndarray:
    """Zero-mean Gaussian random field with covariance var*exp(-d^2/(2 corr^2))
    on the interior nodes, sampled exactly by circulant embedding on a
    periodic grid of twice the domain (negative embedding eigenvalues, which
    are round-off sized here, are clipped to zero)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 2.0 * l / (n + 1)
    m = 2 * (n + 1)
    j = np.arange(m)
    d = np.minimum(j, m - j) * h
    c = var * np.exp(-0.5 * (d / corr) ** 2)
    lam = np.clip(np.fft.fft(c).real, 0.0, None)
    z = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    y = np.fft.fft(np.sqrt(lam / m) * z)
    return np.ascontiguousarray(y.real[:n])


def log_minmax(g: np.ndarray, lo: float, hi: float) -> np.ndarray:
    """exp(g) mapped onto [lo, hi] by an affine map of its logarithm."""
    gmin, gmax = float(g.min()), float(g.max())
    return np.exp(math.log(lo) + (g - gmin) / (gmax - gmin) * (math.log(hi) - math.log(lo)))


def sigmoid(v):
    return 1.0 / (1.0 + np.exp(-v))


@dataclass
class Problem:
    """One instance of Eq. (1.1) on Omega = (-l, l), t in (0, T]."""
    name: str
    alpha: float
    gamma: float
    l: float
    T: float
    r: float
    n: int
    M: int
    soe_tol: float = 1e-12
    krylov_tol: float = 1e-12
    mu: Optional[float] = None
    kappa_mu: Optional[int] = None
    phi: np.ndarray = None
    kappa0: np.ndarray = None
    kappa1: Optional[np.ndarray] = None
    theta: Optional[Callable[[float], float]] = None
    F: list = field(default_factory=list)
    G: list = field(default_factory=list)
    kappa_fn: Optional[Callable] = None
    f_fn: Optional[Callable] = None
    exact: Optional[Callable] = None

    @property
    def x(self) -> np.ndarray:
        return interior_nodes(self.n, self.l)

    @property
    def separable(self) -> bool:
        return self.kappa_fn is None and self.f_fn is None

    def kappa_at(self, t: float) -> np.ndarray:
        if self.kappa_fn is not None:
            return np.asarray(self.kappa_fn(self.x, t), dtype=np.float64)
        k = self.kappa0.copy()
        if self.kappa1 is not None:
            k = k + self.theta(t) * self.kappa1
        return k

    def f_at(self, t: float) -> np.ndarray:
        if self.f_fn is not None:
            return np.asarray(self.f_fn(self.x, t), dtype=np.float64)
        f = np.zeros(self.n)
        for Fr, Gr in zip(self.F, self.G):
            f = f + Gr(t) * Fr
        return f

    def kappa_table(self, times) -> np.ndarray:
        return np.stack([self.kappa_at(float(t)) for t in times])

    def f_table(self, times) -> np.ndarray:
        return np.stack([self.f_at(float(t)) for t in times])

    def theta_values(self, times) -> Optional[np.ndarray]:
        if self.kappa1 is None:
            return None
        return np.array([self.theta(float(t)) for t in times])

    def G_values(self, times) -> np.ndarray:
        return np.array([[Gr(float(t)) for t in times] for Gr in self.G])

    def exact_table(self, times) -> np.ndarray:
        return np.stack([self.exact(self.x, float(t)) for t in times])


# ---------------------------------------------------------------------------
# The paper's examples (Sec. 5)

def example1(alpha: float, gamma: float, r: float, N: int, M: int, s: int = 3,
             mu: Optional[float] = None, kappa_mu: Optional[int] = None,
             soe_tol: float = 1e-10) -> Problem:
    """Example 1: kappa = (1+t) e^{0.8x+1}, u = (1-x^2)^{s+a/2}(t^g + 1);
    paper N intervals -> n = N - 1 unknowns."""
    n = N - 1
    x = interior_nodes(n)
    phi = (1.0 - x * x) ** (s + 0.5 * alpha)
    kx = np.exp(0.8 * x + 1.0)
    lap = frac_lap_bump(alpha, s, x)
    g1 = math.gamma(1.0 + gamma)
    return Problem(
        name=f"example1(a={alpha},g={gamma},r={r},N={N},M={M})", alpha=alpha, gamma=gamma,
        l=1.0, T=1.0, r=r, n=n, M=M, soe_tol=soe_tol, mu=mu, kappa_mu=kappa_mu,
        phi=phi, kappa0=np.zeros(n), kappa1=kx, theta=lambda t: 1.0 + t,
        F=[phi.copy(), kx * lap],
        G=[lambda t: g1, lambda t: (1.0 + t) * (t ** gamma + 1.0)],
        exact=lambda xx, t: (1.0 - xx * xx) ** (s + 0.5 * alpha) * (t ** gamma + 1.0))


def example2(alpha: float, gamma: float, r: float, N: int, M: int,
             soe_tol: float = 1e-9) -> Problem:
    """Example 2: s = 1, kappa = 7[ln(5+2x+t) + cos(x t)]/4 (not separable)."""
    n = N - 1
    s = 1
    x = interior_nodes(n)
    phi = (1.0 - x * x) ** (s + 0.5 * alpha)
    g1 = math.gamma(1.0 + gamma)

    def kfn(xx, t):
        return 7.0 * (np.log(5.0 + 2.0 * xx + t) + np.cos(xx * t)) / 4.0

    def ffn(xx, t):
        return g1 * (1.0 - xx * xx) ** (s + 0.5 * alpha) + kfn(xx, t) * frac_lap_bump(alpha, s, xx) * (t ** gamma + 1.0)

    return Problem(
        name=f"example2(a={alpha},g={gamma},r={r},N={N},M={M})", alpha=alpha, gamma=gamma,
        l=1.0, T=1.0, r=r, n=n, M=M, soe_tol=soe_tol, phi=phi, kappa_fn=kfn, f_fn=ffn,
        exact=lambda xx, t: (1.0 - xx * xx) ** (s + 0.5 * alpha) * (t ** gamma + 1.0))


# ---------------------------------------------------------------------------
# Workload configurations

def config_smallest(n: int = 127, M: int = 64) -> Problem:
    """n = 127, M = 64, gamma = 0.5 (r = (2-g)/g = 3), alpha = 1.5,
    kappa = 1 + 0.5 sin(pi x) e^{-t}, u = (1 + t^g)(1-x^2)_+^{a/2} and the
    source manufactured from it: since (-Delta)^{a/2}(1-x^2)_+^{a/2} = Gamma(a+1),
    f = Gamma(1+g) phi + kappa Gamma(a+1) (1 + t^g)."""
    alpha, gamma = 1.5, 0.5
    x = interior_nodes(n)
    phi = (1.0 - x * x) ** (0.5 * alpha)
    k1 = 0.5 * np.sin(math.pi * x)
    ga = math.gamma(alpha + 1.0)
    g1 = math.gamma(1.0 + gamma)
    return Problem(
        name="smallest", alpha=alpha, gamma=gamma, l=1.0, T=1.0, r=(2.0 - gamma) / gamma,
        n=n, M=M, soe_tol=1e-12, krylov_tol=1e-12, phi=phi, kappa0=np.ones(n), kappa1=k1,
        theta=lambda t: math.exp(-t),
        F=[phi.copy(), ga * np.ones(n), ga * k1],
        G=[lambda t: g1, lambda t: 1.0 + t ** gamma, lambda t: math.exp(-t) * (1.0 + t ** gamma)],
        exact=lambda xx, t: (1.0 + t ** gamma) * (1.0 - xx * xx) ** (0.5 * alpha))


def config_mid(gamma: float, alpha: float, n: int = 16383, M: int = 2048,
               kappa_seed: int = 1, f_seed: int = 2) -> Problem:
    """n = 2^14 - 1, M = 2048, r = (2-g)/g, kappa = 1 + 0.9 sigmoid(F(x))(1+t)
    with a seeded 16-mode Fourier series F, phi = (1-x^2)^{a/2}, f a seeded
    Fourier field (time independent)."""
    x = interior_nodes(n)
    k1 = 0.9 * sigmoid(fourier_field(n, kappa_seed))
    return Problem(
        name=f"mid(g={gamma},a={alpha})", alpha=alpha, gamma=gamma, l=1.0, T=1.0,
        r=(2.0 - gamma) / gamma, n=n, M=M, phi=(1.0 - x * x) ** (0.5 * alpha),
        kappa0=np.ones(n), kappa1=k1, theta=lambda t: 1.0 + t,
        F=[fourier_field(n, f_seed)], G=[lambda t: 1.0])


def config_mixed(n: int = 131071, M: int = 4096) -> Problem:
    """n = 2^17 - 1, M = 4096, gamma = 0.4 (r = 4), alpha = 1.6, kappa = exp of
    a Gaussian random field (corr 0.1, var 0.5, seed 3) mapped onto [0.2, 5],
    time independent; phi = (1-x^2)^{0.8}; f a Fourier field (seed 4)."""
    alpha, gamma = 1.6, 0.4
    x = interior_nodes(n)
    kap = log_minmax(gaussian_field(n, 3), 0.2, 5.0)
    return Problem(
        name="mixed", alpha=alpha, gamma=gamma, l=1.0, T=1.0, r=(2.0 - gamma) / gamma,
        n=n, M=M, phi=(1.0 - x * x) ** (0.5 * alpha), kappa0=kap, kappa1=None,
        F=[fourier_field(n, 4)], G=[lambda t: 1.0])


def batched_instance_params(B: int = 512, seed: int = 4242):
    """Per-instance (n, alpha, gamma) for the batched workload: n drawn
    log-uniformly from [2^9-1, 2^14-1], alpha ~ U(0.6, 1.9), gamma ~ U(0.2, 0.9)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.floor(np.exp(rng.uniform(math.log(511), math.log(16383), B))).astype(int)
    alphas = rng.uniform(0.6, 1.9, B)
    gammas = rng.uniform(0.2, 0.9, B)
    return ns, alphas, gammas


def config_batched_instance(i: int, n: int, alpha: float, gamma: float, M: int = 1024) -> Problem:
    """Instance i of the batched workload: kappa as in the mixed workload with
    seed 1000 + i, phi = (1-x^2)^{a/2}, f a Fourier field (seed 2000 + i)."""
    x = interior_nodes(n)
    kap = log_minmax(gaussian_field(n, 1000 + i), 0.2, 5.0)
    return Problem(
        name=f"batched[{i}]", alpha=float(alpha), gamma=float(gamma), l=1.0, T=1.0,
        r=(2.0 - gamma) / gamma, n=int(n), M=M, phi=(1.0 - x * x) ** (0.5 * alpha),
        kappa0=kap, kappa1=None, F=[fourier_field(n, 2000 + i)], G=[lambda t: 1.0])


def config_adjoint(n: int = 4095, M: int = 1024, kappa_seed: int = 5, f_seed: int = 6,
                   obs_kappa_seed: int = 7):
    """n = 2^12 - 1, M = 1024, gamma = 0.5 (r = 3), alpha = 1.4,
    time-independent lognormal kappa(x) = exp(GRF) (seed 5), f a Fourier field
    (seed 6), phi = (1-x^2)_+^{a/2}.  Returns (problem, kappa_obs) where
    kappa_obs (seed 7) generates the observation u_obs = u^M(kappa_obs)."""
    alpha, gamma = 1.4, 0.5
    x = interior_nodes(n)
    kap = np.exp(gaussian_field(n, kappa_seed))
    kobs = np.exp(gaussian_field(n, obs_kappa_seed))
    p = Problem(
        name="adjoint", alpha=alpha, gamma=gamma, l=1.0, T=1.0, r=(2.0 - gamma) / gamma,
        n=n, M=M, phi=(1.0 - x * x) ** (0.5 * alpha), kappa0=kap, kappa1=None,
        F=[fourier_field(n, f_seed)], G=[lambda t: 1.0])
    return p, kobs
