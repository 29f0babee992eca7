"""GPU parity of the cluster engine: the mixed level solve with its FP32
inner PBiCGSTAB on one thread-block cluster (FFTs held in distributed
shared memory) against the oracle, against the grid engine, and at the
full workload size on sampled rows."""
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


def test_engine_selection(torch):
    assert solver(n=1023, precision="mixed").engine == "grid"
    assert solver(n=1023, precision="mixed", engine="cluster").engine == "cluster"
    assert solver(n=1023, precision="fp64", engine="cluster").engine == "grid"
    assert solver(n=131071, M=4, precision="mixed", engine="cluster").engine == "cluster"


# sizes span every cluster shape: Q = 1 (n <= 3), 2, 4, 8, 16 CTAs, one to
# sixteen columns and row units per CTA, one- to three-stage FFTs
@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 63, 100, 127, 255, 1000, 1023, 2047])
@pytest.mark.parametrize("a", [1.0e3, 18.0])
def test_cluster_linear_solve_matches_dense_lu(torch, n, a):
    alpha = 1.6
    s = solver(alpha=alpha, n=n, precision="mixed", engine="cluster")
    t = oracle.ifl_symbol(alpha, n)
    kap = ti.log_minmax(ti.gaussian_field(n, 3), 0.2, 5.0) if n > 1 else np.array([1.3])
    b = np.random.default_rng(5).standard_normal(n) * 10
    ref = oracle.lu_solve(a * np.eye(n) + kap[:, None] * oracle.dense_A(t), b)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = s.linear_solve(a, cuda(torch, kap), cuda(torch, b), x)
    err = np.max(np.abs(x.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err < 1e-10, (err, info)
    assert info["status"] == 0 and info["iterations"] > 0


def test_cluster_without_preconditioner(torch):
    n, a, alpha = 255, 50.0, 1.5
    s = solver(alpha=alpha, n=n, precision="mixed", precond="none", engine="cluster")
    t = oracle.ifl_symbol(alpha, n)
    kap = 1.0 + 0.5 * np.sin(np.pi * ti.interior_nodes(n))
    b = np.random.default_rng(9).standard_normal(n)
    ref = oracle.lu_solve(a * np.eye(n) + kap[:, None] * oracle.dense_A(t), b)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.linear_solve(a, cuda(torch, kap), cuda(torch, b), x)
    assert np.max(np.abs(x.cpu().numpy() - ref)) / np.max(np.abs(ref)) < 1e-10


def test_cluster_smallest_config_parity(torch):
    """n = 127, M = 64 march, cluster engine, oracle's SOE table: max relative
    error vs the oracle's dense-LU FIDS <= 1e-10 over all levels."""
    import paper_2002_11978_gb300 as pkg
    prob = ti.config_smallest()
    tm, tau = oracle.graded_mesh(prob.T, prob.M, prob.r)
    soe = oracle.soe_build(prob.gamma, tau[1], prob.T, prob.soe_tol)
    s = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, prob.n, prob.M, prob.r, prob.soe_tol,
                   precision="mixed", soe=soe, krylov_tol=prob.krylov_tol, engine="cluster")
    s.set_problem_from(prob)
    U = torch.zeros((prob.M + 1, prob.n), dtype=torch.float64, device="cuda")
    uf = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    info = s.solve(uf, U)
    assert info["status"] == 0, info
    ref = oracle.march("FIDS", prob.alpha, prob.gamma, prob.l, prob.T, prob.r, prob.n, prob.M,
                       prob.phi, prob.kappa_table(tm), prob.f_table(tm), soe=soe)
    err = np.max(np.abs(U.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err < 1e-10, (err, info)


@pytest.mark.parametrize("n", [4095, 16383])
def test_cluster_matches_grid_engine(torch, n):
    """Same level solves on both engines (both converge to their own
    tolerance): the solutions agree to the requested accuracy."""
    alpha, a = 1.3, 40.0
    kap = ti.log_minmax(ti.gaussian_field(n, 11), 0.2, 5.0)
    b = np.random.default_rng(12).standard_normal(n)
    xs = []
    for eng in ("grid", "cluster"):
        s = solver(alpha=alpha, n=n, precision="mixed", engine=eng)
        assert s.engine == eng
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        info = s.linear_solve(a, cuda(torch, kap), cuda(torch, b), x)
        assert info["status"] == 0, info
        xs.append(x.cpu().numpy())
    assert np.max(np.abs(xs[0] - xs[1])) / np.max(np.abs(xs[0])) < 1e-10


def _sampled_residual(t, a, kap, u, b, rows):
    """max_i |b_i - (a u_i + kap_i (A u)_i)| / max|b| over sampled rows i, with
    row i of the symmetric Toeplitz A summed directly (O(n) per row)."""
    n = len(u)
    worst = 0.0
    for i in rows:
        Au = np.dot(t[np.abs(i - np.arange(n))], u)
        worst = max(worst, abs(b[i] - (a * u[i] + kap[i] * Au)))
    return worst / np.max(np.abs(b))


def test_full_size_levels_mixed_vs_fp64(torch):
    """The full workload (n = 2^17 - 1, M = 4096), first 6 levels: mixed
    (cluster engine) and FP64 agree to 1e-10 relative, and each level's
    solution satisfies its own equation on 64 sampled rows, checked with the
    oracle's symbol."""
    import paper_2002_11978_gb300 as pkg
    prob = ti.config_mixed()
    n, levels = prob.n, 6
    t = oracle.ifl_symbol(prob.alpha, n)
    rows = np.random.default_rng(0).choice(n, 64, replace=False)
    rows[:2] = [0, n - 1]
    sols = {}
    for prec in ("fp64", "mixed"):
        s = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, n, prob.M, prob.r, prob.soe_tol,
                       precision=prec, krylov_tol=prob.krylov_tol,
                       engine="cluster" if prec == "mixed" else "auto")
        if prec == "mixed":
            assert s.engine == "cluster"
        s.set_problem_from(prob)
        u = torch.zeros(n, dtype=torch.float64, device="cuda")
        rhs = torch.zeros(n, dtype=torch.float64, device="cuda")
        out = []
        for m in range(1, levels + 1):
            info = s.step(u_out=u, rhs_out=rhs)
            assert info["status"] == 0, info
            out.append((u.cpu().numpy().copy(), rhs.cpu().numpy().copy()))
        sols[prec] = out
    for (u64, b64), (umx, bmx) in zip(sols["fp64"], sols["mixed"]):
        assert np.max(np.abs(umx - u64)) / np.max(np.abs(u64)) < 1e-10
    # each mixed level solves (ahat_m I + diag(kappa) A) u = rhs
    for m, (umx, bmx) in enumerate(sols["mixed"], start=1):
        ahat_m = oracle.l1_weight(prob.T, prob.M, prob.r, prob.gamma, m, m) / math.gamma(1 - prob.gamma)
        assert _sampled_residual(t, ahat_m, prob.kappa0, umx, bmx, rows) < 1e-9


@pytest.mark.parametrize("gamma", [0.3, 0.7])
@pytest.mark.parametrize("alpha", [0.8, 1.2, 1.8])
def test_mid_size_levels_fp64_mixed_and_sampled_rows(torch, gamma, alpha):
    """The mid workload (n = 2^14 - 1, M = 2048, six (gamma, alpha) pairs),
    first 12 levels: FP64 and mixed agree to 1e-10, and the last level's
    solution satisfies its equation on 64 sampled rows summed with the
    oracle's symbol."""
    import paper_2002_11978_gb300 as pkg
    prob = ti.config_mid(gamma, alpha)
    n, levels = prob.n, 12
    t = oracle.ifl_symbol(prob.alpha, n)
    tm, _ = oracle.graded_mesh(prob.T, prob.M, prob.r)
    rows = np.random.default_rng(1).choice(n, 64, replace=False)
    rows[:2] = [0, n - 1]
    out = {}
    for prec in ("fp64", "mixed"):
        s = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, n, prob.M, prob.r, prob.soe_tol,
                       precision=prec, krylov_tol=prob.krylov_tol)
        s.set_problem_from(prob)
        u = torch.zeros(n, dtype=torch.float64, device="cuda")
        rhs = torch.zeros(n, dtype=torch.float64, device="cuda")
        for m in range(1, levels + 1):
            info = s.step(u_out=u, rhs_out=rhs)
            assert info["status"] == 0, info
        out[prec] = (u.cpu().numpy(), rhs.cpu().numpy())
    u64, umx = out["fp64"][0], out["mixed"][0]
    assert np.max(np.abs(umx - u64)) / np.max(np.abs(u64)) < 1e-10
    ahat = oracle.l1_weight(prob.T, prob.M, prob.r, prob.gamma, levels, levels) / math.gamma(1 - prob.gamma)
    kap = prob.kappa_at(tm[levels])
    assert _sampled_residual(t, ahat, kap, umx, out["mixed"][1], rows) < 1e-9
