"""Residual certificates of GPU marches at full size, where dense LU is out
of reach (the mid workload n = 2^14 - 1, M = 2048, and the headline
n = 2^17 - 1, M = 4096).

For a sampled level m the oracle forms the level's right-hand side b^m from
the GPU's own levels u^0..u^{m-1} with the direct FIDS weights of
Eq. (3.16gu) (the GPU's SOE table), and the defect
d^m = b^m - (ahat_m u^m + kappa^m .* (A u^m)) in double-double arithmetic
(a plain FP64 sum would carry errors ~1e-16 ||A|| ||u||, ~1e-9 of u here).
By Theorem 3.1 the level matrix has diagonal-dominance excess >= ahat_m, so
by Lemma 3.3 ||M^{-1} y|| <= ||y|| / ahat_m.  ||d^m|| / ahat_m alone cannot
go below eps ||M|| / ahat_m ~ 1e-8 at the late headline levels for any FP64
vector; oracle.certify sharpens it with an approximate correction e
(M e ~ d, by numpy FFTs) and the double-double defect of e:
||u_exact^m - u^m|| <= ||e|| + ||d - M e|| / ahat_m (+ rounding terms),
asserted <= 1e-10 max|u^m|.  It covers both the Krylov solve and the SOE
recurrence that formed the GPU's history.

The Toeplitz entries are the context's own (tsfde_get_symbol), checked
against the oracle's to 3e-16 each: at n = 2^17 - 1 the smallest eigenvalue
of A, its row-sum excess ~0.11, is a difference of entries up to ~1e8, so
one-ulp differences between two equally accurate evaluations of the entries
move it by ~1e-9 relative; the certificate is of the level equation the GPU
holds, whose entries are the paper's formula to rounding."""
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
    t = s.symbol()
    t_or = oracle.ifl_symbol(prob.alpha, prob.n)
    assert np.max(np.abs(t - t_or) / np.abs(t_or)) <= 5e-16  # two ulps
    return t, U.cpu().numpy(), s.soe(), s.times()


def certify(prob, t, U, soe, tm, levels):
    """Certified bounds on ||u_exact^m - u^m||_inf relative to max|u^m|, and
    the Lemma 3.3 bounds ||d^m||_inf / ahat_m (relative too) beside them."""
    from oracle import certify as oc
    out, lemma = {}, {}
    oracle.set_threads(os.cpu_count() or 1)
    try:
        for m in levels:
            b = oracle.level_rhs("FIDS", prob.alpha, prob.gamma, prob.l, prob.T, prob.r, prob.n, prob.M,
                                 m, U, prob.f_at(tm[m]), soe=soe)
            ahat = oracle.l1_weight(prob.T, prob.M, prob.r, prob.gamma, m, m) / math.gamma(1 - prob.gamma)
            bound, l33 = oc.certify_level(t, ahat, prob.kappa_at(tm[m]), U[m], b)
            um = float(np.max(np.abs(U[m])))
            out[m], lemma[m] = bound / um, l33 / um
    finally:
        oracle.set_threads(1)
    return out, lemma


@pytest.mark.parametrize("gamma,alpha", [(0.3, 0.8), (0.3, 1.2), (0.3, 1.8),
                                         (0.7, 0.8), (0.7, 1.2), (0.7, 1.8)])
def test_mid_workload_certified(torch, gamma, alpha):
    """n = 2^14 - 1, M = 2048, the six (gamma, alpha) pairs, the default
    path (double-single mixed solve, per-level Krylov choice, extrapolated
    start); levels 1, 2, 10, 100, 1000 and M certified."""
    prob = ti.config_mid(gamma, alpha, M=2048)
    t, U, soe, tm = march(torch, prob, precision="mixed_ds", krylov="auto", warm_start="extrapolate")
    bounds, lemma = certify(prob, t, U, soe, tm, [1, 2, 10, 100, 1000, prob.M])
    assert max(bounds.values()) <= 1e-10, (bounds, lemma)


def test_mid_workload_certified_fp64_bicgstab(torch):
    """The paper's solver (FP64 BiCGSTAB, x0 = 0) on one mid pair."""
    prob = ti.config_mid(0.7, 1.8, M=2048)
    t, U, soe, tm = march(torch, prob)
    bounds, lemma = certify(prob, t, U, soe, tm, [1, 2, 10, 100, 1000, prob.M])
    assert max(bounds.values()) <= 1e-10, (bounds, lemma)


def test_headline_workload_certified(torch):
    """n = 2^17 - 1, M = 4096, the benchmark's default path over the whole
    march; levels 1, 2, 16, 64, 2048 and M certified (each defect is an
    O(n^2) double-double sum)."""
    prob = ti.config_mixed()
    t, U, soe, tm = march(torch, prob, precision="mixed_ds", krylov="auto", warm_start="extrapolate")
    bounds, lemma = certify(prob, t, U, soe, tm, [1, 2, 16, 64, 2048, prob.M])
    assert max(bounds.values()) <= 1e-10, (bounds, lemma)
