"""The largest accepted size, n = 2^18 (and the odd 2^18 - 1), for every
level kernel and Krylov method: work items of 1024 elements, so the kernels
run their prefetch-depth-4 instances.  Kept in a file of its own that runs
last, since it is the slowest GPU test."""
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


def _sampled_residual(t, a, kap, u, b, rows):
    n = len(u)
    worst = 0.0
    for i in rows:
        Au = np.dot(t[np.abs(i - np.arange(n))], u)
        worst = max(worst, abs(b[i] - (a * u[i] + kap[i] * Au)))
    return worst / np.max(np.abs(b))


@pytest.mark.parametrize("n", [262144, 262143])
def test_maximum_size_all_level_kernels(torch, n):
    """The largest accepted n (2^18, and the odd 2^18 - 1): work items of 1024
    elements, so the level kernels run their prefetch-depth-4 instances.
    Three levels (x0 = 0) of FP64 BiCGSTAB, FP64 PCG and the double-single
    mixed solve with either method agree to 1e-10, and each level satisfies
    its equation on 32 rows summed directly with the oracle's symbol.
    M = 4096 as in the headline workload: its first levels have ahat ~1e6,
    so b is dominated by ahat u.  (On a 16-level mesh ahat_1 ~ 95 and the
    level is A-dominated: there the direct-sum residual of any FP64 solution
    sits near 1e-8 of max|b| at this n -- 1.0e-8 for a float64 numpy FFT
    solve -- because ||A|| ~ 1.6e8.)"""
    import paper_2002_11978_gb300 as pkg
    prob = ti.config_mixed(n=n)
    t = oracle.ifl_symbol(prob.alpha, n)
    rows = np.random.default_rng(2).choice(n, 32, replace=False)
    rows[:2] = [0, n - 1]
    sols = {}
    for prec, kry in (("fp64", "bicgstab"), ("fp64", "pcg"), ("mixed_ds", "pcg"), ("mixed_ds", "bicgstab")):
        s = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, n, prob.M, prob.r, prob.soe_tol,
                       precision=prec, krylov_tol=prob.krylov_tol, krylov=kry)
        s.set_problem_from(prob)
        u = torch.zeros(n, dtype=torch.float64, device="cuda")
        rhs = torch.zeros(n, dtype=torch.float64, device="cuda")
        for m in range(1, 4):
            info = s.step(u_out=u, rhs_out=rhs)
            assert info["status"] == 0, (prec, kry, info)
            ahat_m = oracle.l1_weight(prob.T, prob.M, prob.r, prob.gamma, m, m) / math.gamma(1 - prob.gamma)
            un, bn = u.cpu().numpy(), rhs.cpu().numpy()
            assert _sampled_residual(t, ahat_m, prob.kappa0, un, bn, rows) < 1e-9, (prec, kry, m)
        sols[(prec, kry)] = un
        s.close()
    ref = sols[("fp64", "bicgstab")]
    for k, v in sols.items():
        assert np.max(np.abs(v - ref)) / np.max(np.abs(ref)) < 1e-10, k
