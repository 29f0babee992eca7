"""Residual certificates of GPU marches at full size, where dense LU is out
of reach (the mid workload n = 2^14 - 1, M = 2048, and the headline
n = 2^17 - 1, M = 4096).

For a sampled level m the oracle forms the level's right-hand side b^m from
the GPU's own levels u^0..u^{m-1} with the direct FIDS weights of
Eq. (3.16gu) (the GPU's SOE table), and the defect
d^m = b^m - (ahat_m u^m + kappa^m .* (A u^m)) in double-double arithmetic
(a plain FP64 sum would carry errors ~1e-16 ||A|| ||u||, ~1e-9 of u here).
By Theorem 3.1 the level matrix has diagonal-dominance excess >= ahat_m, so
by Lemma 3.3 the GPU level is within ||d^m||_inf / ahat_m of the exact
solution of that level's equation: the per-step bound asserted below to be
<= 1e-10 max|u^m|.  It covers both the Krylov solve and the SOE recurrence
that formed the GPU's history."""
import math
import os

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


def march(torch, prob, levels=None, **kw):
    import paper_2002_11978_gb300 as pkg
    s = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, prob.n, prob.M, prob.r, prob.soe_tol,
                   krylov_tol=1e-12, **kw)
    s.set_problem_from(prob)
    last = prob.M if levels is None else levels
    U = torch.zeros((last + 1, prob.n), dtype=torch.float64, device="cuda")
    s.current_solution(U[0])
    for m in range(1, last + 1):
        s.step(u_out=U[m], sync=False)
    st = s.level_stats(1, last)
    assert all(x["status"] == 0 for x in st), [x for x in st if x["status"]][:3]
    return s, U.cpu().numpy(), s.soe(), s.times()


def certify(prob, U, soe, tm, levels):
    """Per-step bounds ||d^m||_inf / ahat_m relative to max|u^m|."""
    t = oracle.ifl_symbol(prob.alpha, prob.n)
    out = {}
    oracle.set_threads(os.cpu_count() or 1)
    try:
        for m in levels:
            b = oracle.level_rhs("FIDS", prob.alpha, prob.gamma, prob.l, prob.T, prob.r, prob.n, prob.M,
                                 m, U, prob.f_at(tm[m]), soe=soe)
            ahat = oracle.l1_weight(prob.T, prob.M, prob.r, prob.gamma, m, m) / math.gamma(1 - prob.gamma)
            d = oracle.level_defect(t, ahat, prob.kappa_at(tm[m]), U[m], b)
            out[m] = float(np.max(np.abs(d))) / ahat / float(np.max(np.abs(U[m])))
    finally:
        oracle.set_threads(1)
    return out


@pytest.mark.parametrize("gamma,alpha", [(0.3, 0.8), (0.3, 1.2), (0.3, 1.8),
                                         (0.7, 0.8), (0.7, 1.2), (0.7, 1.8)])
def test_mid_workload_certified(torch, gamma, alpha):
    """n = 2^14 - 1, M = 2048, the six (gamma, alpha) pairs, the default
    path (double-single mixed solve, per-level Krylov choice, warm start);
    levels 1, 2, 10, 100, 1000 and M certified."""
    prob = ti.config_mid(gamma, alpha, M=2048)
    s, U, soe, tm = march(torch, prob, precision="mixed_ds", krylov="auto", warm_start=True)
    bounds = certify(prob, U, soe, tm, [1, 2, 10, 100, 1000, prob.M])
    assert max(bounds.values()) <= 1e-10, bounds


def test_mid_workload_certified_fp64_bicgstab(torch):
    """The paper's solver (FP64 BiCGSTAB, x0 = 0) on one mid pair."""
    prob = ti.config_mid(0.7, 1.8, M=2048)
    s, U, soe, tm = march(torch, prob)
    bounds = certify(prob, U, soe, tm, [1, 2, 10, 100, 1000, prob.M])
    assert max(bounds.values()) <= 1e-10, bounds


def test_headline_workload_certified(torch):
    """n = 2^17 - 1, M = 4096, the benchmark's default path over the whole
    march; levels 1, 2, 16, 64, 2048 and M certified (each defect is an
    O(n^2) double-double sum)."""
    prob = ti.config_mixed()
    s, U, soe, tm = march(torch, prob, precision="mixed_ds", krylov="auto", warm_start=True)
    bounds = certify(prob, U, soe, tm, [1, 2, 16, 64, 2048, prob.M])
    assert max(bounds.values()) <= 1e-10, bounds
