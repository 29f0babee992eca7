"""GPU parity of the double-single path (precision TSFDE_MIXED_DS): the
Toeplitz product in double-single arithmetic against the oracle's direct
product, and the mixed level solves with a double-single inner PBiCGSTAB
against dense LU, the oracle's march and the FP64 path."""
import math

import numpy as np
import pytest

import oracle
import tsfde_inputs as ti

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2002_11978_gb300 import build
    build.build()
    return T


def cuda(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def solver(alpha=1.5, gamma=0.5, n=127, M=8, r=3.0, **kw):
    import paper_2002_11978_gb300 as pkg
    return pkg.Solver(alpha, gamma, 1.0, 1.0, n, M, r, kw.pop("soe_tol", 1e-12), **kw)


def _L(n):
    return max(8, 1 << math.ceil(math.log2(max(2 * n - 1, 1))))


# ------------------------------------------------------------- products
@pytest.mark.parametrize("n", [1, 2, 3, 7, 127, 128, 1000, 4095, 16383])
@pytest.mark.parametrize("alpha", [0.5, 1.5, 1.9])
def test_toeplitz_apply_double_single_matches_dense(torch, n, alpha):
    """y = A v (Sec. 4.1) with the FFT in double-single: normwise error
    against the oracle's direct sum within a few 2^-48 per FFT stage."""
    s = solver(alpha=alpha, n=n, precision="mixed_ds")
    t = oracle.ifl_symbol(alpha, n)
    v = np.random.default_rng(n).standard_normal(n)
    ref = oracle.toeplitz_matvec(t, v)
    scale = (t[0] + 2 * np.sum(np.abs(t[1:]))) * np.max(np.abs(v))
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.toeplitz_apply(cuda(torch, v), y, "mixed_ds")
    err = np.max(np.abs(y.cpu().numpy() - ref)) / scale
    assert err < 2e-14 * math.log2(_L(n)) * 4, err


def test_double_single_product_needs_its_context(torch):
    import paper_2002_11978_gb300 as pkg
    s = solver(n=31)
    v = torch.ones(31, dtype=torch.float64, device="cuda")
    y = torch.zeros(31, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.TsfdeError) as e:
        s.toeplitz_apply(v, y, "mixed_ds")
    assert e.value.status == pkg.TSFDE_EINVAL


@pytest.mark.parametrize("n", [1023, 4095, 16383])
def test_product_resolves_low_modes_of_rough_input(torch, n):
    """For white v, y = v + A v is dominated by its high frequencies and its
    low modes sit far below |y|.  The error that matters to the
    preconditioned solve is the one seen through the Strang preconditioner
    P = I + s(A) (Eq. (4.3)): |P^{-1}(y - y_ref)| / |P^{-1} y_ref|, with P
    applied as a circulant (numpy FFT) and y_ref the oracle's direct sum.
    Double-single stays within 1e-9 of it; FP32 is over 100x worse."""
    alpha = 1.6
    t = oracle.ifl_symbol(alpha, n)
    lam = np.fft.fft(oracle.strang_column(t)).real
    pinv = lambda x: np.fft.ifft(np.fft.fft(x) / (1.0 + lam)).real
    v = np.random.default_rng(11).standard_normal(n)
    ref = v + oracle.toeplitz_matvec(t, v)
    pr = np.max(np.abs(pinv(ref)))
    s = solver(alpha=alpha, n=n, precision="mixed_ds")
    ones = cuda(torch, np.ones(n))
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    errs = {}
    for prec in ("fp64", "mixed_ds", "fp32"):
        s.operator_apply(1.0, ones, cuda(torch, v), y, prec)
        errs[prec] = np.max(np.abs(pinv(y.cpu().numpy() - ref))) / pr
    assert errs["fp64"] < 1e-11, errs
    assert errs["mixed_ds"] < 1e-9, errs
    assert errs["fp32"] > 100 * errs["mixed_ds"], errs


@pytest.mark.parametrize("n", [7, 127, 1000])
def test_precond_apply_double_single(torch, n):
    """P^{-1} v built in FP64, rounded and applied in double-single, vs
    dense LU of the circulant (Eq. (4.3))."""
    alpha = 1.5
    s = solver(alpha=alpha, n=n, precision="mixed_ds")
    t = oracle.ifl_symbol(alpha, n)
    c = oracle.strang_column(t)
    C = c[(np.arange(n)[:, None] - np.arange(n)[None, :]) % n]
    a, kbar = 25.0, 1.7
    v = np.random.default_rng(3).standard_normal(n)
    ref = oracle.lu_solve(a * np.eye(n) + kbar * C, v)
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.precond_apply(a, kbar, cuda(torch, v), z, "mixed_ds")
    assert np.max(np.abs(z.cpu().numpy() - ref)) / np.max(np.abs(ref)) < 1e-11


# ---------------------------------------------------------- level solves
@pytest.mark.parametrize("n", [1, 2, 63, 127, 1023])
@pytest.mark.parametrize("a", [1.0e3, 18.0])
def test_linear_solve_double_single_matches_dense_lu(torch, n, a):
    alpha = 1.6
    s = solver(alpha=alpha, n=n, precision="mixed_ds")
    t = oracle.ifl_symbol(alpha, n)
    kap = ti.log_minmax(ti.gaussian_field(n, 3), 0.2, 5.0) if n > 2 else np.full(n, 1.3)
    b = np.random.default_rng(5).standard_normal(n) * 10
    ref = oracle.lu_solve(a * np.eye(n) + kap[:, None] * oracle.dense_A(t), b)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = s.linear_solve(a, cuda(torch, kap), cuda(torch, b), x)
    err = np.max(np.abs(x.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err < 1e-10, (err, info)
    assert info["status"] == 0 and info["outer"] > 0, info


def test_linear_solve_double_single_without_preconditioner(torch):
    n, a, alpha = 127, 50.0, 1.5
    s = solver(alpha=alpha, n=n, precision="mixed_ds", precond="none")
    t = oracle.ifl_symbol(alpha, n)
    kap = 1.0 + 0.5 * np.sin(np.pi * ti.interior_nodes(n))
    b = np.random.default_rng(9).standard_normal(n)
    ref = oracle.lu_solve(a * np.eye(n) + kap[:, None] * oracle.dense_A(t), b)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.linear_solve(a, cuda(torch, kap), cuda(torch, b), x)
    assert np.max(np.abs(x.cpu().numpy() - ref)) / np.max(np.abs(ref)) < 1e-10


def _march(torch, prob, precision, soe, **kw):
    import paper_2002_11978_gb300 as pkg
    s = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, prob.n, prob.M, prob.r, prob.soe_tol,
                   precision=precision, soe=soe, krylov_tol=prob.krylov_tol, **kw)
    s.set_problem_from(prob)
    U = torch.zeros((prob.M + 1, prob.n), dtype=torch.float64, device="cuda")
    uf = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    info = s.solve(uf, U)
    assert info["status"] == 0, info
    return U.cpu().numpy(), info


@pytest.mark.parametrize("warm", [False, True, "extrapolate"])
def test_smallest_config_march_matches_oracle(torch, warm):
    """n = 127, M = 64 with the oracle's SOE table: every level within 1e-10
    of the oracle's FIDS march (direct history sums, dense LU)."""
    prob = ti.config_smallest()
    tm, tau = oracle.graded_mesh(prob.T, prob.M, prob.r)
    soe = oracle.soe_build(prob.gamma, tau[1], prob.T, prob.soe_tol)
    U, info = _march(torch, prob, "mixed_ds", soe, warm_start=warm)
    ref = oracle.march("FIDS", prob.alpha, prob.gamma, prob.l, prob.T, prob.r, prob.n, prob.M,
                       prob.phi, prob.kappa_table(tm), prob.f_table(tm), soe=soe)
    err = np.max(np.abs(U - ref)) / np.max(np.abs(ref))
    assert err < 1e-10, (err, info)


def _sampled_residual(t, a, kap, u, b, rows):
    n = len(u)
    worst = 0.0
    for i in rows:
        Au = np.dot(t[np.abs(i - np.arange(n))], u)
        worst = max(worst, abs(b[i] - (a * u[i] + kap[i] * Au)))
    return worst / np.max(np.abs(b))


@pytest.mark.parametrize("warm", [False, True])
def test_full_size_levels_double_single_vs_fp64(torch, warm):
    """n = 2^17 - 1, M = 4096 (spectral range ~1e8), first 6 levels: the
    double-single inner solves resolve the operator, so no level falls back
    to FP64 and the inner iterations stay within 1.5x of FP64's; u agrees
    with FP64 to 1e-10 and satisfies its level equation on 64 rows summed
    directly with the oracle's symbol."""
    import paper_2002_11978_gb300 as pkg
    prob = ti.config_mixed()
    n, levels = prob.n, 6
    t = oracle.ifl_symbol(prob.alpha, n)
    rows = np.random.default_rng(0).choice(n, 64, replace=False)
    rows[:2] = [0, n - 1]
    sols, its = {}, {}
    for prec in ("fp64", "mixed_ds"):
        s = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, n, prob.M, prob.r, prob.soe_tol,
                       precision=prec, krylov_tol=prob.krylov_tol, warm_start=warm)
        s.set_problem_from(prob)
        u = torch.zeros(n, dtype=torch.float64, device="cuda")
        rhs = torch.zeros(n, dtype=torch.float64, device="cuda")
        out, it = [], 0
        for m in range(1, levels + 1):
            info = s.step(u_out=u, rhs_out=rhs)
            assert info["status"] == 0, info
            if prec == "mixed_ds":
                assert info["outer"] >= 0, info  # negative: finished in FP64
            it += info["iterations"]
            out.append((u.cpu().numpy().copy(), rhs.cpu().numpy().copy()))
        sols[prec], its[prec] = out, it
    assert its["mixed_ds"] <= 1.5 * its["fp64"], its
    for (u64, _), (uds, _) in zip(sols["fp64"], sols["mixed_ds"]):
        assert np.max(np.abs(uds - u64)) / np.max(np.abs(u64)) < 1e-10
    for m, (uds, bds) in enumerate(sols["mixed_ds"], start=1):
        ahat_m = oracle.l1_weight(prob.T, prob.M, prob.r, prob.gamma, m, m) / math.gamma(1 - prob.gamma)
        assert _sampled_residual(t, ahat_m, prob.kappa0, uds, bds, rows) < 1e-9


@pytest.mark.parametrize("gamma,alpha", [(0.3, 1.8), (0.7, 0.8)])
def test_mid_size_levels_double_single_vs_fp64(torch, gamma, alpha):
    """n = 2^14 - 1, M = 2048, first 12 levels: double-single mixed agrees
    with FP64 to 1e-10."""
    import paper_2002_11978_gb300 as pkg
    prob = ti.config_mid(gamma, alpha)
    out = {}
    for prec in ("fp64", "mixed_ds"):
        s = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, prob.n, prob.M, prob.r, prob.soe_tol,
                       precision=prec, krylov_tol=prob.krylov_tol)
        s.set_problem_from(prob)
        u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
        for m in range(1, 13):
            assert s.step(u_out=u)["status"] == 0
        out[prec] = u.cpu().numpy()
    assert np.max(np.abs(out["mixed_ds"] - out["fp64"])) / np.max(np.abs(out["fp64"])) < 1e-10
