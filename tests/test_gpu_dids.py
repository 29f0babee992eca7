"""GPU parity of the direct-history scheme DIDS (Eq. (4.1); history =
"direct"): the right-hand side against the direct L1 sum with the oracle's
weights, whole marches against the oracle's DIDS, the printed errors of
Sec. 5, and agreement with FIDS to the SOE tolerance (Thm 3.4 vs 3.5)."""
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


def _solver(prob, precision="fp64", history="direct", **kw):
    import paper_2002_11978_gb300 as pkg
    s = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, prob.n, prob.M, prob.r, prob.soe_tol,
                   precision=precision, krylov_tol=prob.krylov_tol, history=history, **kw)
    s.set_problem_from(prob)
    return s


def test_rhs_is_the_direct_l1_sum(torch):
    """b^m = Gamma(1-g)^{-1}[sum_{k=1}^{m-1}(a_{k+1}-a_k) u^k + a_1 u^0] + f^m
    (Eq. (4.1)), element by element at every level of the smallest config,
    with the GPU's own levels u^k and the oracle's weights a_k^{(m)}."""
    prob = ti.config_smallest()
    s = _solver(prob)
    tm = s.times()
    n, M = prob.n, prob.M
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    rhs = torch.zeros(n, dtype=torch.float64, device="cuda")
    U = [prob.phi.copy()]
    Gg = math.gamma(1.0 - prob.gamma)
    worst = 0.0
    for m in range(1, M + 1):
        s.step(u_out=u, rhs_out=rhs)
        a = [0.0] + [oracle.l1_weight(prob.T, M, prob.r, prob.gamma, m, k) for k in range(1, m + 1)]
        ref = a[1] * U[0]
        for k in range(1, m):
            ref = ref + (a[k + 1] - a[k]) * U[k]
        scale = np.max(a[1] * np.abs(U[0]) + sum(abs(a[k + 1] - a[k]) * np.abs(U[k]) for k in range(1, m)))
        ref = ref / Gg + prob.f_at(tm[m])
        worst = max(worst, np.max(np.abs(rhs.cpu().numpy() - ref)) / (scale / Gg))
        U.append(u.cpu().numpy().copy())
    assert worst < 1e-14, worst


@pytest.mark.parametrize("precision,warm", [("fp64", False), ("fp64", True), ("mixed_ds", False),
                                            ("mixed", False)])
def test_march_matches_oracle_dids(torch, precision, warm):
    """n = 127, M = 64: every level within 1e-10 of the oracle's DIDS march
    (direct L1 sums, dense LU)."""
    prob = ti.config_smallest()
    s = _solver(prob, precision, warm_start=warm)
    U = torch.zeros((prob.M + 1, prob.n), dtype=torch.float64, device="cuda")
    uf = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    info = s.solve(uf, U)
    assert info["status"] == 0, info
    tm, _ = oracle.graded_mesh(prob.T, prob.M, prob.r)
    ref = oracle.march("DIDS", prob.alpha, prob.gamma, prob.l, prob.T, prob.r, prob.n, prob.M,
                       prob.phi, prob.kappa_table(tm), prob.f_table(tm))
    err = np.max(np.abs(U.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err < 1e-10, (err, info)


def _printed(v, p):
    e = math.floor(math.log10(p))
    return abs(v - p) <= 0.55 * 10.0 ** (e - 3)


def _rows():
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append(line.split())
    return rows


ROWS = [r for r in _rows() if r[0] in ("T1", "T3", "T11") and int(r[8]) * int(r[7]) <= 2e4]


@pytest.mark.parametrize("row", ROWS, ids=["-".join(r[:9]) for r in ROWS])
def test_paper_tables_with_direct_history(torch, row):
    """Sec. 5: the GPU DIDS reproduces the printed Err_inf/Err_2 (4 digits)."""
    tab, ex = row[0], int(row[1])
    alpha, r, gamma = float(row[2]), float(row[3]), float(row[4])
    N, M = int(row[7]), int(row[8])
    prob = ti.example1(alpha, gamma, r, N, M) if ex == 1 else ti.example2(alpha, gamma, r, N, M)
    import paper_2002_11978_gb300 as pkg
    s = pkg.Solver(alpha, gamma, 1.0, 1.0, prob.n, M, r, prob.soe_tol, history="direct",
                   krylov_tol=1e-10 if tab == "T11" else 1e-12)
    tm = s.times()
    cu = lambda v: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda")
    if ex == 1:
        s.set_problem_from(prob)
    else:
        s.set_problem(cu(prob.phi), torch.zeros(prob.n, dtype=torch.float64, device="cuda"))
    Uh = np.zeros((M + 1, prob.n))
    Uh[0] = prob.phi
    u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    for m in range(1, M + 1):
        if ex == 1:
            s.step(u_out=u)
        else:
            s.step(kappa_m=cu(prob.kappa_at(tm[m])), f_m=cu(prob.f_at(tm[m])), u_out=u)
        Uh[m] = u.cpu().numpy()
    ei, e2 = oracle.errors(Uh, prob.exact_table(tm), 2.0 / N)
    assert _printed(ei, float(row[9])), (ei, row[9])
    if row[10] != "-":
        assert _printed(e2, float(row[10])), (e2, row[10])


def _levels(torch, prob, history, precision, levels):
    s = _solver(prob, precision, history=history)
    u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    for _ in range(levels):
        assert s.step(u_out=u)["status"] == 0
    return u.cpu().numpy()


def test_dids_equals_fids_mid_size(torch):
    """n = 2^14 - 1, M = 2048 (soe_tol 1e-12), first 48 levels: DIDS and FIDS
    agree to 1e-10 relative (they differ by the SOE error, Thm 3.4 vs 3.5)."""
    prob = ti.config_mid(0.3, 1.8)
    ud = _levels(torch, prob, "direct", "fp64", 48)
    uf = _levels(torch, prob, "soe", "fp64", 48)
    assert np.max(np.abs(ud - uf)) / np.max(np.abs(uf)) < 1e-10


def test_dids_equals_fids_full_size(torch):
    """n = 2^17 - 1, M = 4096 (all levels held: 4.3 GB), first 6 levels with
    the double-single mixed solve: DIDS and FIDS agree to 1e-10."""
    prob = ti.config_mixed()
    ud = _levels(torch, prob, "direct", "mixed_ds", 6)
    uf = _levels(torch, prob, "soe", "mixed_ds", 6)
    assert np.max(np.abs(ud - uf)) / np.max(np.abs(uf)) < 1e-10


def test_adjoint_needs_the_soe_history(torch):
    import paper_2002_11978_gb300 as pkg
    prob = ti.config_smallest(n=31, M=4)
    prob.kappa1 = None
    s = _solver(prob)
    U = torch.zeros((prob.M + 1, prob.n), dtype=torch.float64, device="cuda")
    uf = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    s.solve(uf, U)
    g = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.TsfdeError) as e:
        s.adjoint(U, torch.ones(prob.n, dtype=torch.float64, device="cuda"), g, g.clone())
    assert e.value.status == pkg.TSFDE_ENOTSUP
