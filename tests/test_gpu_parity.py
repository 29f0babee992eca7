"""GPU parity: every operation of the FIDS hot path, through the C ABI,
against the CPU oracle on the same seeded inputs."""
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


# ------------------------------------------------------ Toeplitz product
@pytest.mark.parametrize("n", [1, 2, 3, 7, 127, 128, 1000, 4095, 16383])
@pytest.mark.parametrize("alpha", [0.5, 1.5, 1.9])
def test_toeplitz_apply_matches_dense(torch, n, alpha):
    s = solver(alpha=alpha, n=n)
    t = oracle.ifl_symbol(alpha, n)
    np.testing.assert_allclose(s.symbol(), t, rtol=1e-14, atol=0)
    v = np.random.default_rng(n).standard_normal(n)
    ref = oracle.toeplitz_matvec(t, v)
    scale = (t[0] + 2 * np.sum(np.abs(t[1:]))) * np.max(np.abs(v))
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.toeplitz_apply(cuda(torch, v), y, "fp64")
    err64 = np.max(np.abs(y.cpu().numpy() - ref)) / scale
    s.toeplitz_apply(cuda(torch, v), y, "fp32")
    err32 = np.max(np.abs(y.cpu().numpy() - ref)) / scale
    L = max(8, 1 << math.ceil(math.log2(max(2 * n - 1, 1))))
    assert err64 < 4e-16 * math.log2(L) * 4, err64
    assert err32 < 2e-7 * math.log2(L) * 4, err32


@pytest.mark.parametrize("n", [5, 127, 1023])
def test_operator_apply_matches_dense(torch, n):
    s = solver(alpha=1.2, n=n)
    t = oracle.ifl_symbol(1.2, n)
    rng = np.random.default_rng(7)
    v = rng.standard_normal(n)
    kap = np.exp(rng.standard_normal(n))
    a = 37.5
    ref = a * v + kap * oracle.toeplitz_matvec(t, v)
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.operator_apply(a, cuda(torch, kap), cuda(torch, v), y, "fp64")
    scale = (a + np.max(kap) * (t[0] + 2 * np.sum(np.abs(t[1:])))) * np.max(np.abs(v))
    assert np.max(np.abs(y.cpu().numpy() - ref)) / scale < 1e-14


# --------------------------------------------------- Strang preconditioner
@pytest.mark.parametrize("n", [1, 2, 7, 8, 127, 128, 255, 1000])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_precond_apply_matches_dense_circulant(torch, n, prec):
    """z = (a I + kbar s(A))^{-1} v, Eq. (4.3), vs dense LU of the circulant."""
    alpha = 1.5
    s = solver(alpha=alpha, n=n)
    t = oracle.ifl_symbol(alpha, n)
    c = oracle.strang_column(t)
    C = c[(np.arange(n)[:, None] - np.arange(n)[None, :]) % n]
    a, kbar = 25.0, 1.7
    v = np.random.default_rng(3).standard_normal(n)
    ref = oracle.lu_solve(a * np.eye(n) + kbar * C, v)
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.precond_apply(a, kbar, cuda(torch, v), z, prec)
    err = np.max(np.abs(z.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err < (1e-11 if prec == "fp64" else 2e-4), err


# ------------------------------------------------------- level solves
@pytest.mark.parametrize("n", [63, 127, 1023])
@pytest.mark.parametrize("a", [1.0e3, 18.0])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_linear_solve_matches_dense_lu(torch, n, a, precision):
    alpha = 1.6
    s = solver(alpha=alpha, n=n, precision=precision)
    t = oracle.ifl_symbol(alpha, n)
    kap = ti.log_minmax(ti.gaussian_field(n, 3), 0.2, 5.0)
    b = np.random.default_rng(5).standard_normal(n) * 10
    ref = oracle.lu_solve(a * np.eye(n) + kap[:, None] * oracle.dense_A(t), b)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = s.linear_solve(a, cuda(torch, kap), cuda(torch, b), x)
    err = np.max(np.abs(x.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err < 1e-10, (err, info)
    assert info["status"] == 0 and info["iterations"] > 0


def test_linear_solve_without_preconditioner(torch):
    n, a, alpha = 127, 50.0, 1.5
    s = solver(alpha=alpha, n=n, precond="none")
    t = oracle.ifl_symbol(alpha, n)
    kap = 1.0 + 0.5 * np.sin(np.pi * ti.interior_nodes(n))
    b = np.random.default_rng(9).standard_normal(n)
    ref = oracle.lu_solve(a * np.eye(n) + kap[:, None] * oracle.dense_A(t), b)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = s.linear_solve(a, cuda(torch, kap), cuda(torch, b), x)
    assert np.max(np.abs(x.cpu().numpy() - ref)) / np.max(np.abs(ref)) < 1e-10
    s2 = solver(alpha=alpha, n=n)
    info2 = s2.linear_solve(a, cuda(torch, kap), cuda(torch, b), x)
    assert info2["iterations"] < info["iterations"]


# ------------------------------------------------------ time marching
def _oracle_fids(prob, soe, mu=None, kappa_mu=None):
    tm, _ = oracle.graded_mesh(prob.T, prob.M, prob.r)
    return oracle.march("FIDS", prob.alpha, prob.gamma, prob.l, prob.T, prob.r, prob.n, prob.M,
                        prob.phi, prob.kappa_table(tm), prob.f_table(tm), mu=mu,
                        kappa_mu=kappa_mu, soe=soe)


def _gpu_solve(torch, prob, precision="fp64", soe=None, **kw):
    import paper_2002_11978_gb300 as pkg
    s = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, prob.n, prob.M, prob.r, prob.soe_tol,
                   precision=precision, soe=soe, krylov_tol=prob.krylov_tol, **kw)
    s.set_problem_from(prob)
    U = torch.zeros((prob.M + 1, prob.n), dtype=torch.float64, device="cuda")
    uf = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    info = s.solve(uf, U)
    assert info["status"] == 0, info
    np.testing.assert_array_equal(uf.cpu().numpy(), U[-1].cpu().numpy())
    return s, U.cpu().numpy(), info


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_smallest_config_parity_same_soe_table(torch, precision):
    """n = 127, M = 64: GPU FIDS (SOE recurrence, FFT products, PBiCGSTAB at
    tol 1e-12) vs oracle FIDS (direct history sums, dense LU), both with
    the oracle's SOE table: max relative error <= 1e-10 over all levels."""
    prob = ti.config_smallest()
    tm, tau = oracle.graded_mesh(prob.T, prob.M, prob.r)
    soe = oracle.soe_build(prob.gamma, tau[1], prob.T, prob.soe_tol)
    _, U, info = _gpu_solve(torch, prob, precision, soe=soe)
    ref = _oracle_fids(prob, soe)
    err = np.max(np.abs(U - ref)) / np.max(np.abs(ref))
    assert err < 1e-10, (err, info)


def test_smallest_config_parity_own_soe_table(torch):
    """The library's compressed SOE table also meets the parity bar against
    the oracle's plain trapezoid table (both within soe_tol = 1e-12)."""
    prob = ti.config_smallest()
    tm, tau = oracle.graded_mesh(prob.T, prob.M, prob.r)
    s, U, info = _gpu_solve(torch, prob, "fp64")
    ss, ww = s.soe()
    assert oracle.soe_rel_err(prob.gamma, tau[1], prob.T, ss, ww) <= prob.soe_tol
    assert info["E"] == len(ss)
    ref = _oracle_fids(prob, oracle.soe_build(prob.gamma, tau[1], prob.T, prob.soe_tol))
    err = np.max(np.abs(U - ref)) / np.max(np.abs(ref))
    assert err < 1e-10, err
    # distance to the exact PDE solution is the scheme's discretisation
    # error, the same for GPU and oracle
    ex = prob.exact_table(tm)
    assert abs(np.max(np.abs(U - ex)) - np.max(np.abs(ref - ex))) < 1e-10


def test_rhs_history_recurrence_matches_direct_sums(torch):
    """The SOE recurrence for the history (a2) gives the same right-hand side
    as the direct FIDS sum of Eq. (3.16gu) with the oracle's b_k weights,
    evaluated on the GPU's own solution history."""
    import paper_2002_11978_gb300 as pkg
    prob = ti.config_smallest(n=63, M=24)
    tm, tau = oracle.graded_mesh(prob.T, prob.M, prob.r)
    soe = oracle.soe_build(prob.gamma, tau[1], prob.T, prob.soe_tol)
    s = pkg.Solver(prob.alpha, prob.gamma, 1.0, 1.0, prob.n, prob.M, prob.r, prob.soe_tol, soe=soe)
    s.set_problem_from(prob)
    U = [prob.phi.copy()]
    u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    rhs = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    Gg = math.gamma(1 - prob.gamma)
    worst = 0.0
    for m in range(1, prob.M + 1):
        s.step(u_out=u, rhs_out=rhs)
        c = [None] + [oracle.fids_weight(prob.T, prob.M, prob.r, prob.gamma, m, k, *soe) for k in range(1, m + 1)]
        ref = c[1] * U[0]
        for k in range(1, m):
            ref = ref + (c[k + 1] - c[k]) * U[k]
        ref = ref / Gg + prob.f_at(tm[m])
        worst = max(worst, np.max(np.abs(rhs.cpu().numpy() - ref)) / np.max(np.abs(ref)))
        U.append(u.cpu().numpy())
    assert worst < 1e-12, worst


@pytest.mark.parametrize("n,M", [(1, 1), (1, 5), (2, 3), (3, 7), (5, 2)])
def test_edge_sizes(torch, n, M):
    prob = ti.config_smallest(n=n, M=M)
    tm, tau = oracle.graded_mesh(prob.T, prob.M, prob.r)
    soe = oracle.soe_build(prob.gamma, tau[1], prob.T, prob.soe_tol)
    _, U, _ = _gpu_solve(torch, prob, "fp64", soe=soe)
    ref = _oracle_fids(prob, soe)
    assert np.max(np.abs(U - ref)) / np.max(np.abs(ref)) < 1e-10


def test_step_after_last_level_is_a_state_error(torch):
    import paper_2002_11978_gb300 as pkg
    prob = ti.config_smallest(n=15, M=2)
    s = pkg.Solver(prob.alpha, prob.gamma, 1.0, 1.0, prob.n, prob.M, prob.r, 1e-12)
    s.set_problem_from(prob)
    s.step()
    s.step()
    with pytest.raises(pkg.TsfdeError) as e:
        s.step()
    assert e.value.status == pkg.TSFDE_ESTATE
    s.reset()
    assert s.step()["m"] == 1


# ------------------------------------------------------------ paper tables
def _table_rows():
    import os
    rows = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            rows.append(f)
    return rows


def _printed(v, p):
    e = math.floor(math.log10(p))
    return abs(v - p) <= 0.55 * 10.0 ** (e - 3)


PAPER_GPU_ROWS = [r for r in _table_rows() if r[0] in ("T1", "T5", "T7", "T9", "T11")
                  and int(r[8]) * int(r[7]) <= 2e5]


@pytest.mark.parametrize("row", PAPER_GPU_ROWS, ids=["-".join(r[:9]) for r in PAPER_GPU_ROWS])
def test_paper_tables_on_gpu(torch, row):
    """Sec. 5 Tables: the GPU FIDS reproduces the printed Err_inf/Err_2 (4
    digits); Table 11 rows also check the average PBiCGSTAB iteration count
    per level against the printed FIDS+P value (the paper counts in half
    iterations: allowed difference 1)."""
    import paper_2002_11978_gb300 as pkg
    tab, ex = row[0], int(row[1])
    alpha, r, gamma = float(row[2]), float(row[3]), float(row[4])
    mu = None if row[5] == "d" else float(row[5])
    kmu = int(row[6]) if mu else None
    N, M = int(row[7]), int(row[8])
    prob = (ti.example1(alpha, gamma, r, N, M, mu=mu, kappa_mu=kmu) if ex == 1
            else ti.example2(alpha, gamma, r, N, M))
    s = pkg.Solver(alpha, gamma, 1.0, 1.0, prob.n, M, r, prob.soe_tol, mu=mu, kappa_mu=kmu,
                   krylov_tol=1e-10 if tab == "T11" else 1e-12)
    tm = s.times()
    if ex == 1:
        s.set_problem_from(prob)
    else:
        z = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
        s.set_problem(cuda(torch, prob.phi), z)
    U = np.zeros((M + 1, prob.n))
    U[0] = prob.phi
    u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    its = 0
    for m in range(1, M + 1):
        if ex == 1:
            info = s.step(u_out=u)
        else:
            info = s.step(kappa_m=cuda(torch, prob.kappa_at(tm[m])), f_m=cuda(torch, prob.f_at(tm[m])), u_out=u)
        its += info["iterations"]
        U[m] = u.cpu().numpy()
    ei, e2 = oracle.errors(U, prob.exact_table(tm), 2.0 / N)
    assert _printed(ei, float(row[9])), (ei, row[9])
    if row[10] != "-":
        assert _printed(e2, float(row[10])), (e2, row[10])
    if row[11] != "-":
        assert abs(its / M - float(row[11])) <= 1.0, (its / M, row[11])


@pytest.mark.parametrize("warm", [True, "extrapolate"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_warm_start_march_matches_oracle(torch, precision, warm):
    """Levels started from u^{m-1}, or from the cubic extrapolation through
    u^{m-4} .. u^{m-1} (stopping at ||r|| < tol ||b||), reach the same
    solutions as the oracle's dense-LU march."""
    prob = ti.config_smallest()
    tm, tau = oracle.graded_mesh(prob.T, prob.M, prob.r)
    soe = oracle.soe_build(prob.gamma, tau[1], prob.T, prob.soe_tol)
    _, U, info = _gpu_solve(torch, prob, precision, soe=soe, warm_start=warm)
    ref = _oracle_fids(prob, soe)
    assert np.max(np.abs(U - ref)) / np.max(np.abs(ref)) < 1e-10, info


def test_warm_start_large_levels_agree(torch):
    """n = 16383: 24 levels with and without warm start (u^{m-1} or the
    extrapolated start), FP64 and mixed."""
    import paper_2002_11978_gb300 as pkg
    prob = ti.config_mid(0.3, 1.8, n=16383, M=64)
    out = {}
    for prec in ("fp64", "mixed"):
        for warm in (False, True, "extrapolate"):
            s = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, prob.n, prob.M, prob.r, prob.soe_tol,
                           precision=prec, warm_start=warm)
            s.set_problem_from(prob)
            u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
            for _ in range(24):
                info = s.step(u_out=u)
                assert info["status"] == 0, info
            out[(prec, warm)] = u.cpu().numpy()
    ref = out[("fp64", False)]
    for k, v in out.items():
        assert np.max(np.abs(v - ref)) / np.max(np.abs(ref)) < 1e-10, k


def test_barrier_timeout_returns_status_and_context_survives(torch):
    """A barrier that gives up at once (timeout of 1 cycle) turns into
    TSFDE_ETIMEOUT from the level solve -- no hang, no trap -- and a fresh
    context on the same device works afterwards."""
    import paper_2002_11978_gb300 as pkg
    prob = ti.config_smallest(n=63, M=4)
    s = pkg.Solver(prob.alpha, prob.gamma, 1.0, 1.0, prob.n, prob.M, prob.r, 1e-12,
                   barrier_timeout_cycles=1)
    s.set_problem_from(prob)
    with pytest.raises(pkg.TsfdeError) as e:
        s.step()
    assert e.value.status == pkg.TSFDE_ETIMEOUT
    torch.cuda.synchronize()
    s2 = pkg.Solver(prob.alpha, prob.gamma, 1.0, 1.0, prob.n, prob.M, prob.r, 1e-12)
    s2.set_problem_from(prob)
    assert s2.step()["status"] == 0


def test_nonfinite_input_is_reported(torch):
    """A NaN in the right-hand side is reported as TSFDE_ENONFINITE."""
    import paper_2002_11978_gb300 as pkg
    n = 127
    s = solver(n=n)
    kap = np.ones(n)
    b = np.ones(n)
    b[5] = np.nan
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.TsfdeError) as e:
        s.linear_solve(10.0, cuda(torch, kap), cuda(torch, b), x)
    assert e.value.status == pkg.TSFDE_ENONFINITE
