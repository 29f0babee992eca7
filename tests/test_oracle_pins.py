"""Pins for the CPU oracle against what the paper and mathematics fix.

None of these re-type an oracle formula: each compares the oracle with a
closed form, an exact identity, a high-precision (50-digit decimal)
evaluation of the defining expression, a library routine, or a value printed
in the paper.
"""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest
from scipy import integrate

import oracle
import tsfde_inputs as ti

getcontext().prec = 50


# ---------------------------------------------------------------- Eq. (1.4)
def test_c1alpha_alpha1_is_one_over_pi():
    assert oracle.c1alpha(1.0) == pytest.approx(1.0 / math.pi, rel=1e-15)


@pytest.mark.parametrize("alpha", [0.3, 0.7, 1.3, 1.8])
def test_c1alpha_normalises_fourier_symbol(alpha):
    # (-Delta)^{a/2} e^{i x} = e^{i x}  <=>  2 c_{1,a} int_0^inf (1-cos y) y^{-1-a} dy = 1
    # [0,1]: (1-cos y)/y^2 is smooth; the y^{1-a} factor goes into the
    # algebraic quadrature weight.  [1,inf): int y^{-1-a} = 1/a and a
    # Fourier-weighted rule for the cosine part.
    g = lambda y: 2.0 * (math.sin(0.5 * y) / y) ** 2 if y > 0 else 0.5
    head, _ = integrate.quad(g, 0.0, 1.0, weight="alg", wvar=(1.0 - alpha, 0.0), epsabs=0, epsrel=1e-13)
    tail2, _ = integrate.quad(lambda y: y ** (-1.0 - alpha), 1.0, np.inf, weight="cos", wvar=1.0)
    I = head + 1.0 / alpha - tail2
    assert 2.0 * oracle.c1alpha(alpha) * I == pytest.approx(1.0, rel=1e-9)


# ------------------------------------------------------------- Eq. (3.16x)
CASES = [(0.4, None), (0.5, None), (1.0, None), (1.5, None), (1.9, None), (1.6, 2.0), (0.4, 2.0)]


def _C(alpha, mu, n, l=1.0):
    nu = mu - alpha
    h = 2.0 * l / (n + 1)
    return oracle.c1alpha(alpha) / (nu * h ** alpha)


@pytest.mark.parametrize("alpha,mu", CASES)
@pytest.mark.parametrize("n", [1, 2, 3, 7, 64, 255])
def test_symbol_prop31_structure(alpha, mu, n):
    """Prop. 3.1: a_11 > 0, off-diagonals negative with strictly decaying
    magnitude, strict diagonal dominance with the proof's explicit margins."""
    km = None if mu is None else 2
    t = oracle.ifl_symbol(alpha, n, mu=mu, kappa_mu=km)
    mu_ = 1 + alpha / 2 if mu is None else mu
    km_ = 1 if mu is None else 2
    nu = mu_ - alpha
    N = n + 1
    C = _C(alpha, mu_, n)
    assert t[0] > 0
    if n > 1:
        assert np.all(t[1:] < 0)
        assert np.all(np.diff(np.abs(t)) < 0) and t[0] > abs(t[1])
    A = oracle.dense_A(t)
    excess = np.diag(A) - (np.sum(np.abs(A), axis=1) - np.abs(np.diag(A)))
    tail = (N ** nu - (N - 1) ** nu) / N ** mu_ + 2 * nu / (alpha * N ** alpha)
    assert excess[0] > C * ((2 ** nu + km_ - 1) / 2 + tail) * (1 - 1e-12) or n == 1
    assert np.all(excess > C * tail * (1 - 1e-12))
    assert np.allclose(A, A.T)
    assert np.all(np.linalg.eigvalsh(A) > 0)


@pytest.mark.parametrize("alpha,mu", [(1.5, None), (0.5, None), (1.9, None), (1.6, 2.0)])
def test_symbol_entries_vs_50_digit_decimal(alpha, mu):
    """t_k / C against a 50-digit evaluation of the bracket of Eq. (3.16x),
    including large k where the plain difference of powers cancels."""
    n = 4095
    km = 1 if mu is None else 2
    mu_ = 1 + alpha / 2 if mu is None else mu
    t = oracle.ifl_symbol(alpha, n, mu=mu, kappa_mu=km if mu is not None else None)
    C = _C(alpha, mu_, n)
    nu = Decimal(repr(mu_ - alpha))
    muD = Decimal(repr(mu_))
    for k in [2, 3, 17, 500, 4094]:
        K = Decimal(k)
        ref = -((K + 1) ** nu - (K - 1) ** nu) / (2 * K ** muD)
        assert t[k] / C == pytest.approx(float(ref), rel=2e-14)
    ref1 = -(Decimal(2) ** nu + km - 1) / 2
    assert t[1] / C == pytest.approx(float(ref1), rel=1e-15)


@pytest.mark.parametrize("alpha,mu", [(1.5, None), (0.5, None), (1.6, 2.0)])
def test_symbol_diagonal_vs_50_digit_decimal(alpha, mu):
    n = 200
    N = n + 1
    km = 1 if mu is None else 2
    mu_ = 1 + alpha / 2 if mu is None else mu
    t = oracle.ifl_symbol(alpha, n, mu=mu, kappa_mu=km if mu is not None else None)
    nu = Decimal(repr(mu_ - alpha))
    muD = Decimal(repr(mu_))
    aD = Decimal(repr(alpha))
    s = sum(((Decimal(l) + 1) ** nu - (Decimal(l) - 1) ** nu) / Decimal(l) ** muD for l in range(2, N))
    ND = Decimal(N)
    ref = s + (ND ** nu - (ND - 1) ** nu) / ND ** muD + (Decimal(2) ** nu + km - 1) + 2 * nu / (aD * ND ** aD)
    assert t[0] / _C(alpha, mu_, n) == pytest.approx(float(ref), rel=1e-14)


@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.5, 1.9])
def test_symbol_second_order_on_smooth_bump(alpha):
    """Lemma 2.4 / Remark 3.1: for u = (1-x^2)_+^{3+a/2} (s = 3) and
    mu = 1 + a/2 the discrete IFL converges at O(h^2) to the closed form
    2^a Gamma((a+1)/2) Gamma(s+1+a/2)/(sqrt(pi) Gamma(s+1)) 2F1((a+1)/2,-s;1/2;x^2)."""
    errs = []
    for n in [127, 255, 511]:
        x = ti.interior_nodes(n)
        t = oracle.ifl_symbol(alpha, n)
        Au = oracle.toeplitz_matvec(t, (1 - x * x) ** (3 + alpha / 2))
        ex = ti.frac_lap_bump(alpha, 3, x)
        errs.append(np.max(np.abs(Au - ex)[np.abs(x) <= 0.5]))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.95) and np.all(rates < 2.15)
    assert errs[-1] < 2e-4


@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.5, 1.9])
def test_symbol_bump_s0_gamma_alpha_plus_1(alpha):
    """(-Delta)^{a/2}(1-x^2)_+^{a/2} = Gamma(a+1) on Omega; the discrete
    operator converges to it (observed order ~1 + a/2 in the interior)."""
    errs = []
    for n in [255, 511, 1023]:
        x = ti.interior_nodes(n)
        t = oracle.ifl_symbol(alpha, n)
        Au = oracle.toeplitz_matvec(t, (1 - x * x) ** (alpha / 2))
        errs.append(np.max(np.abs(Au - math.gamma(alpha + 1))[np.abs(x) <= 0.5]))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 0.9 * (1 + alpha / 2) - 0.1)
    assert errs[-1] < 1e-3


# ------------------------------------------------------------ graded mesh
@pytest.mark.parametrize("M,r", [(64, 3.0), (4096, 4.0), (1024, 1.0), (2048, 2.0 / 0.3 - 1.0)])
def test_graded_mesh_vs_decimal(M, r):
    t, tau = oracle.graded_mesh(1.0, M, r)
    assert t[M] == 1.0 and t[0] == 0.0
    rD = Decimal(repr(r))
    MD = Decimal(M)
    for k in [1, 2, 3, M // 2, M - 1, M]:
        ref = (Decimal(k) / MD) ** rD - (Decimal(k - 1) / MD) ** rD if k > 1 else (Decimal(1) / MD) ** rD
        assert tau[k] == pytest.approx(float(ref), rel=4e-15)
    assert math.fsum(tau) == pytest.approx(1.0, rel=1e-14)
    for (m, k) in [(M, 1), (M, M - 1), (3, 2), (M // 2 + 1, M // 2)]:
        ref = (Decimal(m) / MD) ** rD - (Decimal(k) / MD) ** rD
        assert oracle.lib().or_mesh_gap(1.0, M, r, m, k) == pytest.approx(float(ref), rel=4e-15)


# ------------------------------------------------------------ Eq. (2.8)
def _a_decimal(M, r, gamma, m, k):
    rD = Decimal(repr(r))
    g1 = 1 - Decimal(repr(gamma))
    tD = lambda j: (Decimal(j) / Decimal(M)) ** rD
    tau = tD(k) - tD(k - 1)
    hi = (tD(m) - tD(k - 1)) ** g1
    lo = (tD(m) - tD(k)) ** g1 if m > k else Decimal(0)
    return (hi - lo) / (g1 * tau)


@pytest.mark.parametrize("M,r,gamma", [(64, 3.0, 0.5), (4096, 4.0, 0.4), (1024, 1.0, 0.8)])
def test_l1_weights_vs_decimal(M, r, gamma):
    for (m, k) in [(M, 1), (M, 2), (M, M // 2), (M, M - 1), (M, M), (2, 1), (7, 3), (M // 3, 1)]:
        a = oracle.l1_weight(1.0, M, r, gamma, m, k)
        assert a == pytest.approx(float(_a_decimal(M, r, gamma, m, k)), rel=3e-14), (m, k)


@pytest.mark.parametrize("M,r,gamma", [(64, 3.0, 0.5), (512, 4.0, 0.4)])
def test_l1_exact_for_ramps(M, r, gamma):
    """The L1 formula is exact for piecewise-linear u: for u = (t - t_j)_+ the
    Caputo derivative at t_m is (t_m-t_j)^{1-g}/Gamma(2-g), i.e.
    sum_{k>j} a_k^{(m)} tau_k = (t_m - t_j)^{1-g}/(1-g)."""
    t, tau = oracle.graded_mesh(1.0, M, r)
    for m in [1, 2, M // 2, M]:
        a = np.array([oracle.l1_weight(1.0, M, r, gamma, m, k) for k in range(1, m + 1)])
        for j in sorted({0, m // 3, m - 1}):
            lhs = math.fsum(a[j:] * tau[j + 1:m + 1])
            gap = oracle.lib().or_mesh_gap(1.0, M, r, m, j)
            assert lhs == pytest.approx(gap ** (1 - gamma) / (1 - gamma), rel=1e-13)


# ------------------------------------------------------------ Lemma 2.2
@pytest.mark.parametrize("gamma,M,r,tol", [(0.5, 64, 3.0, 1e-12), (0.4, 4096, 4.0, 1e-12),
                                           (0.8, 256, 3.0, 1e-10), (0.2, 1024, 9.0, 1e-9)])
def test_soe_bound(gamma, M, r, tol):
    delta = M ** (-r)
    s, w = oracle.soe_build(gamma, delta, 1.0, tol)
    assert np.all(s > 0) and np.all(w > 0)
    # independent check at random points with numpy
    rng = np.random.default_rng(0)
    tt = np.exp(rng.uniform(math.log(delta), 0.0, 3000))
    approx = np.array([np.sum(w * np.exp(-s * t1)) for t1 in tt])
    assert np.max(np.abs(tt ** gamma * approx - 1)) <= tol


@pytest.mark.parametrize("gamma,M,r", [(0.5, 64, 3.0), (0.4, 256, 4.0)])
def test_fids_weights_within_soe_tolerance_of_l1(gamma, M, r):
    """b_k^{(m)} integrates the SOE kernel over [t_{k-1}, t_k] where a_k^{(m)}
    integrates (t_m - s)^{-g}; a relative kernel error <= eps gives
    |b_k - a_k| <= eps a_k."""
    tol = 1e-10
    s, w = oracle.soe_build(gamma, M ** (-r), 1.0, tol)
    for m in [2, M // 2, M]:
        for k in sorted({1, 2, m // 2, m - 1}):
            a = oracle.l1_weight(1.0, M, r, gamma, m, k)
            b = oracle.fids_weight(1.0, M, r, gamma, m, k, s, w)
            assert abs(b - a) <= 1.01 * tol * a
        assert oracle.fids_weight(1.0, M, r, gamma, m, m, s, w) == oracle.l1_weight(1.0, M, r, gamma, m, m)


# --------------------------------------------------- dense linear algebra
def test_lu_matches_lapack_and_known_solution():
    rng = np.random.default_rng(1)
    for n in [1, 2, 5, 40]:
        A = rng.standard_normal((n, n)) + np.diag(rng.uniform(0, 0.1, n))
        x = rng.standard_normal(n)
        b = A @ x
        xs = oracle.lu_solve(A, b)
        assert np.allclose(xs, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)
        assert np.allclose(xs, x, rtol=1e-8, atol=1e-9)
    P = np.array([[0.0, 1.0], [1.0, 0.0]])  # needs pivoting
    assert np.allclose(oracle.lu_solve(P, np.array([2.0, 3.0])), [3.0, 2.0])


def test_toeplitz_matvec_matches_dense_product():
    rng = np.random.default_rng(2)
    t = rng.standard_normal(33)
    v = rng.standard_normal(33)
    assert np.allclose(oracle.toeplitz_matvec(t, v), oracle.dense_A(t) @ v, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------- Sec. 4.1 Strang
@pytest.mark.parametrize("n", [1, 2, 6, 7, 63, 127, 128])
def test_strang_column_and_eigenvalues(n):
    t = oracle.ifl_symbol(1.5, n)
    c = oracle.strang_column(t)
    # circulant whose first column is c must be symmetric: c_k = c_{n-k}
    assert np.allclose(c[1:], c[1:][::-1], rtol=0, atol=0)
    # and it must copy the central band of A: c_k = t_k for k <= n/2
    assert np.array_equal(c[: n // 2 + 1], t[: n // 2 + 1])
    lam = oracle.strang_eigs(t)
    assert np.allclose(lam, np.fft.fft(c).real, rtol=1e-12, atol=1e-12 * t[0])
    # Lemma 4.1: all eigenvalues in (0, 2 a_11)
    assert np.all(lam > 0) and np.all(lam < 2 * t[0])


# ------------------------------------------------------- Tables 1-11
def _load_rows():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        rows.append(dict(table=f[0], ex=int(f[1]), alpha=float(f[2]), r=float(f[3]), gamma=float(f[4]),
                         mu=None if f[5] == "d" else float(f[5]), kappa_mu=int(f[6]), N=int(f[7]),
                         M=int(f[8]), err_inf=None if f[9] == "-" else float(f[9]),
                         err_2=None if f[10] == "-" else float(f[10]),
                         its_P=None if f[11] == "-" else float(f[11]),
                         its_I=None if f[12] == "-" else float(f[12])))
    return rows


PAPER_ROWS = _load_rows()


def paper_problem(row):
    if row["ex"] == 1:
        return ti.example1(row["alpha"], row["gamma"], row["r"], row["N"], row["M"],
                           mu=row["mu"], kappa_mu=row["kappa_mu"] if row["mu"] else None)
    return ti.example2(row["alpha"], row["gamma"], row["r"], row["N"], row["M"])


def printed_match(v, p):
    """v rounds to the 4-significant-digit printed value p."""
    e = math.floor(math.log10(p))
    return abs(v - p) <= 0.55 * 10.0 ** (e - 3)


def run_oracle(row, scheme):
    p = paper_problem(row)
    tm, tau = oracle.graded_mesh(p.T, p.M, p.r)
    soe = oracle.soe_build(p.gamma, tau[1], p.T, p.soe_tol) if scheme == "FIDS" else None
    U = oracle.march(scheme, p.alpha, p.gamma, p.l, p.T, p.r, p.n, p.M, p.phi,
                     p.kappa_table(tm), p.f_table(tm), mu=p.mu,
                     kappa_mu=p.kappa_mu if p.mu else None, soe=soe)
    return p, tm, U


@pytest.mark.parametrize("scheme", ["DIDS", "FIDS"])
@pytest.mark.parametrize("row", PAPER_ROWS, ids=[f"{r['table']}-{r['N']}-{r['M']}-{r['r']}-{r['gamma']}-{r['alpha']}" for r in PAPER_ROWS])
def test_paper_table_errors(row, scheme):
    """Err_inf / Err_2 of Sec. 5 reproduced to the printed 4 digits."""
    if row["M"] * row["M"] * row["N"] > 2e8 and scheme == "FIDS":
        pytest.skip("covered by DIDS; FIDS-direct history is O(M^2 E) per run")
    p, tm, U = run_oracle(row, scheme)
    ei, e2 = oracle.errors(U, p.exact_table(tm), 2.0 / row["N"])
    assert printed_match(ei, row["err_inf"]), (ei, row["err_inf"])
    if row["err_2"] is not None:
        assert printed_match(e2, row["err_2"]), (e2, row["err_2"])


def test_fids_equals_dids_to_soe_tolerance():
    """Thm 3.4 vs 3.5: FIDS differs from DIDS by O(eps)."""
    p = ti.config_smallest()
    tm, tau = oracle.graded_mesh(p.T, p.M, p.r)
    K, F = p.kappa_table(tm), p.f_table(tm)
    soe = oracle.soe_build(p.gamma, tau[1], p.T, 1e-12)
    Ud = oracle.march("DIDS", p.alpha, p.gamma, p.l, p.T, p.r, p.n, p.M, p.phi, K, F)
    Uf = oracle.march("FIDS", p.alpha, p.gamma, p.l, p.T, p.r, p.n, p.M, p.phi, K, F, soe=soe)
    assert np.max(np.abs(Uf - Ud)) / np.max(np.abs(Ud)) < 1e-10


def test_stability_bound_thm31x():
    """||u^k|| <= ||u^0|| + Gamma(1-g) max_s ||f^s|| / b_1^{(s)}."""
    p = ti.config_smallest(n=63, M=32)
    tm, tau = oracle.graded_mesh(p.T, p.M, p.r)
    soe = oracle.soe_build(p.gamma, tau[1], p.T, 1e-12)
    F = p.f_table(tm)
    U = oracle.march("FIDS", p.alpha, p.gamma, p.l, p.T, p.r, p.n, p.M, p.phi, p.kappa_table(tm), F, soe=soe)
    Gg = math.gamma(1 - p.gamma)
    for k in range(1, p.M + 1):
        bound = np.max(np.abs(U[0])) + Gg * max(
            np.max(np.abs(F[s])) / oracle.fids_weight(p.T, p.M, p.r, p.gamma, s, 1, *soe) for s in range(1, k + 1))
        assert np.max(np.abs(U[k])) <= bound


def test_temporal_order_smallest_config():
    """Thm 3.4 with spatial error frozen out: O(M^{-min(r g, 2-g)}) = O(M^{-1.5})
    for g = 0.5, r = 3; measured against a reference run at 4M."""
    base = ti.config_smallest(n=15, M=16)
    errs = []
    ref = None
    for M in [16, 32, 64, 256]:
        p = ti.config_smallest(n=15, M=M)
        tm, _ = oracle.graded_mesh(p.T, p.M, p.r)
        U = oracle.march("DIDS", p.alpha, p.gamma, p.l, p.T, p.r, p.n, p.M, p.phi,
                         p.kappa_table(tm), p.f_table(tm))
        errs.append(U[-1])
    ref = errs[-1]
    e = [np.max(np.abs(u - ref)) for u in errs[:-1]]
    rates = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert np.all(rates > 1.2), rates
    del base


# ---------------------------------------------------------------- adjoint
def test_adjoint_matches_central_differences():
    """Dense adjoint gradients vs central differences of J through the
    oracle's own forward march (h = 1e-6, random directions)."""
    n, M = 15, 12
    prob, kobs = ti.config_adjoint(n=n, M=M)
    tm, tau = oracle.graded_mesh(prob.T, M, prob.r)
    soe = oracle.soe_build(prob.gamma, tau[1], prob.T, 1e-12)
    kap0 = prob.kappa0
    f0 = prob.F[0]
    u_obs = oracle.march("FIDS", prob.alpha, prob.gamma, prob.l, prob.T, prob.r, n, M, prob.phi,
                         np.tile(kobs, (M + 1, 1)), np.tile(f0, (M + 1, 1)), soe=soe)[M]

    def J(kap, f):
        U = oracle.march("FIDS", prob.alpha, prob.gamma, prob.l, prob.T, prob.r, n, M, prob.phi,
                         np.tile(kap, (M + 1, 1)), np.tile(f, (M + 1, 1)), soe=soe)
        return 0.5 * np.sum((U[M] - u_obs) ** 2)

    J0, _, gk, gf = oracle.adjoint(prob.alpha, prob.gamma, prob.l, prob.T, prob.r, n, M, prob.phi,
                                   kap0, f0, u_obs, soe)
    assert J0 == pytest.approx(J(kap0, f0), rel=1e-14)
    rng = np.random.default_rng(11)
    h = 1e-6
    for _ in range(4):
        d = rng.standard_normal(n)
        d /= np.linalg.norm(d)
        fd_k = (J(kap0 + h * d, f0) - J(kap0 - h * d, f0)) / (2 * h)
        fd_f = (J(kap0, f0 + h * d) - J(kap0, f0 - h * d)) / (2 * h)
        assert gk @ d == pytest.approx(fd_k, rel=1e-6, abs=1e-12)
        assert gf @ d == pytest.approx(fd_f, rel=1e-6, abs=1e-12)


def test_threaded_lu_gives_the_same_bits():
    """The timed CPU baseline may run the LU's row updates on several threads;
    each row's update is the same operation sequence, so the solution must be
    bitwise that of one thread."""
    rng = np.random.default_rng(11)
    n = 300
    A = rng.standard_normal((n, n)) + n * np.eye(n)
    b = rng.standard_normal(n)
    x1 = oracle.lu_solve(A, b)
    try:
        oracle.set_threads(4)
        x4 = oracle.lu_solve(A, b)
    finally:
        oracle.set_threads(1)
    assert np.array_equal(x1, x4)
    assert oracle.get_threads() == 1


def test_level_defect_matches_exact_rational_arithmetic():
    """The double-double defect d = b - (a u + kappa .* (A u)) against the
    exact value in rational arithmetic, on a case built to cancel: b is the
    FP64 evaluation of a u + kappa .* (A u), so the exact defect is at the
    rounding level of terms ~1e6 times larger, where a plain FP64
    evaluation returns noise."""
    from fractions import Fraction
    rng = np.random.default_rng(4)
    n = 12
    t = np.concatenate(([3.0e6], -rng.uniform(1e4, 1e5, n - 1)))
    u = rng.standard_normal(n)
    kap = rng.uniform(0.2, 5.0, n)
    a = 17.25
    Au = np.array([sum(t[abs(i - j)] * u[j] for j in range(n)) for i in range(n)])
    b = a * u + kap * Au
    d = oracle.level_defect(t, a, kap, u, b)
    F = Fraction
    for i in range(n):
        s = sum(F(t[abs(i - j)]) * F(u[j]) for j in range(n))
        exact = F(b[i]) - (F(a) * F(u[i]) + F(kap[i]) * s)
        mag = abs(a * u[i]) + kap[i] * sum(abs(t[abs(i - j)] * u[j]) for j in range(n))
        assert abs(F(d[i]) - exact) <= F(2.0 ** -100 * mag) + abs(exact) * F(2.0 ** -52), i
    # the threaded evaluation gives the same bits
    try:
        oracle.set_threads(3)
        assert np.array_equal(oracle.level_defect(t, a, kap, u, b), d)
    finally:
        oracle.set_threads(1)


@pytest.mark.parametrize("scheme", ["FIDS", "DIDS"])
def test_level_rhs_is_the_march_right_hand_side(scheme):
    """level_rhs(m) from the march's own levels 0..m-1 is the right-hand side
    the march solved at level m: its levels satisfy their equations with it
    to rounding, measured by the double-double defect."""
    prob = ti.config_smallest(n=31, M=12)
    tm, tau = oracle.graded_mesh(prob.T, prob.M, prob.r)
    soe = oracle.soe_build(prob.gamma, tau[1], prob.T, prob.soe_tol) if scheme == "FIDS" else None
    K, F = prob.kappa_table(tm), prob.f_table(tm)
    U = oracle.march(scheme, prob.alpha, prob.gamma, prob.l, prob.T, prob.r, prob.n, prob.M, prob.phi,
                     K, F, soe=soe)
    t = oracle.ifl_symbol(prob.alpha, prob.n)
    for m in (1, 2, 7, prob.M):
        b = oracle.level_rhs(scheme, prob.alpha, prob.gamma, prob.l, prob.T, prob.r, prob.n, prob.M, m,
                             U, F[m], soe=soe)
        ahat = oracle.l1_weight(prob.T, prob.M, prob.r, prob.gamma, m, m) / math.gamma(1 - prob.gamma)
        d = oracle.level_defect(t, ahat, K[m], U[m], b)
        assert np.max(np.abs(d)) <= 1e-13 * np.max(np.abs(b)), (m, np.max(np.abs(d)))


def test_certificate_bounds_the_true_error_tightly():
    """oracle.certify: for a level solved by dense LU and then perturbed by a
    known amount, the certified bound must lie above the true error
    (computed against the LU solution, itself accurate to ~1e-14 here) and
    within a factor 2 of it; the Lemma 3.3 bound alone is looser."""
    from oracle import certify
    n, a, alpha = 300, 18.0, 1.6
    t = oracle.ifl_symbol(alpha, n)
    kap = ti.log_minmax(ti.gaussian_field(n, 3), 0.2, 5.0)
    b = np.random.default_rng(2).standard_normal(n) * 10
    u_exact = oracle.lu_solve(a * np.eye(n) + kap[:, None] * oracle.dense_A(t), b)
    for scale in (1e-7, 1e-10):
        du = scale * np.random.default_rng(3).standard_normal(n) * np.max(np.abs(u_exact))
        u = u_exact + du
        bound, lemma = certify.certify_level(t, a, kap, u, b)
        true = np.max(np.abs(u - u_exact))
        # the LU reference carries its own rounding, ~1e-16 of max|u|
        assert true - 1e-14 * np.max(np.abs(u_exact)) <= bound <= 2.0 * true, (scale, true, bound)
        assert lemma >= bound


def test_certificate_of_the_exact_solution_is_at_rounding_level():
    from oracle import certify
    n, a, alpha = 200, 1.0e3, 1.2
    t = oracle.ifl_symbol(alpha, n)
    kap = 1.0 + 0.5 * np.sin(np.pi * ti.interior_nodes(n))
    b = np.random.default_rng(8).standard_normal(n)
    u = oracle.lu_solve(a * np.eye(n) + kap[:, None] * oracle.dense_A(t), b)
    bound, _ = certify.certify_level(t, a, kap, u, b)
    assert bound <= 1e-13 * np.max(np.abs(u)), bound
