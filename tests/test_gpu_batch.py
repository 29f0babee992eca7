"""Batched solve (tsfde_batch_*): many independent FIDS problems in one
persistent launch of thread-block clusters.  Each instance is checked
against the oracle's dense-LU FIDS march at small sizes, and against the
single-problem GPU path (FP64) at the batched workload's sizes, including
its Krylov iteration counts (which a wrong preconditioner would change)."""
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


def _instances(torch, specs, M):
    """specs: list of (i, n, alpha, gamma) -> (instance dicts, problems)."""
    inst, probs = [], []
    for i, n, a, g in specs:
        p = ti.config_batched_instance(i, n, a, g, M=M)
        probs.append(p)
        inst.append(dict(alpha=p.alpha, gamma=p.gamma, n=p.n, r=p.r, phi=cuda(torch, p.phi),
                         kappa=cuda(torch, p.kappa0), f=cuda(torch, p.F[0])))
    return inst, probs


def _batch(torch, inst, M, **kw):
    import paper_2002_11978_gb300 as pkg
    bs = pkg.BatchSolver(inst, M, **kw)
    outs = [torch.zeros(d["n"], dtype=torch.float64, device="cuda") for d in inst]
    info = bs.solve(outs)
    return bs, [u.cpu().numpy() for u in outs], info


def _single(torch, p, precision="fp64"):
    import paper_2002_11978_gb300 as pkg
    s = pkg.Solver(p.alpha, p.gamma, p.l, p.T, p.n, p.M, p.r, 1e-12, precision=precision)
    s.set_problem(cuda(torch, p.phi), cuda(torch, p.kappa0), None, None, F=[cuda(torch, p.F[0])],
                  G=[np.ones(p.M + 1)])
    uf = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    info = s.solve(uf)
    assert info["status"] == 0, info
    return uf.cpu().numpy(), info


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("krylov", ["bicgstab", "pcg", "auto"])
def test_batch_matches_oracle(torch, precision, krylov):
    """Five instances of different n, alpha, gamma (cluster sizes from 4 to
    8 CTAs' worth of rows), M = 12: each u^M against the oracle's dense FIDS
    march with its plain SOE table (both tables within 1e-12), with the
    paper's BiCGSTAB or PCG on the symmetrised system (ce_pcg)."""
    M = 12
    specs = [(0, 63, 1.5, 0.5), (1, 127, 0.8, 0.3), (2, 200, 1.9, 0.8), (3, 511, 1.2, 0.6),
             (4, 96, 0.6, 0.2)]
    inst, probs = _instances(torch, specs, M)
    bs, U, info = _batch(torch, inst, M, precision=precision, krylov=krylov)
    assert info["status"] == 0 and info["iterations"] > 0, info
    for p, u in zip(probs, U):
        tm, tau = oracle.graded_mesh(p.T, M, p.r)
        soe = oracle.soe_build(p.gamma, tau[1], p.T, 1e-12)
        ref = oracle.march("FIDS", p.alpha, p.gamma, p.l, p.T, p.r, p.n, M, p.phi,
                           np.tile(p.kappa0, (M + 1, 1)), np.tile(p.F[0], (M + 1, 1)), soe=soe)[M]
        err = np.max(np.abs(u - ref)) / np.max(np.abs(ref))
        assert err < 1e-10, (p.n, err)


def test_batch_matches_single_problem_path(torch):
    """Instances at the batched workload's sizes (n up to 2^14 - 1), M = 8,
    FP64 on both sides: same u^M, same preconditioned iteration counts."""
    M = 8
    specs = [(10, 16383, 1.7, 0.4), (11, 4095, 0.9, 0.7), (12, 1023, 1.3, 0.25), (13, 511, 1.85, 0.5)]
    inst, probs = _instances(torch, specs, M)
    bs, U, info = _batch(torch, inst, M, precision="fp64")
    assert info["status"] == 0, info
    for k, (p, u) in enumerate(zip(probs, U)):
        ref, sinfo = _single(torch, p)
        assert np.max(np.abs(u - ref)) / np.max(np.abs(ref)) < 1e-10
        its = bs.instance_stats(k)["iterations"]
        assert abs(its - sinfo["iterations"]) <= 0.15 * sinfo["iterations"] + 2, (its, sinfo)


def test_batch_mixed_matches_fp64(torch):
    """Mixed precision (FP32 sweeps, FP64 refinement) against FP64 on a
    sample of the batched workload's instances, M = 32."""
    M = 32
    ns, al, ga = ti.batched_instance_params()
    specs = [(i, int(ns[i]), float(al[i]), float(ga[i])) for i in (0, 5, 17, 42, 99, 311)]
    inst, probs = _instances(torch, specs, M)
    _, Um, im = _batch(torch, inst, M, precision="mixed")
    _, Ud, idd = _batch(torch, inst, M, precision="fp64")
    assert im["status"] == 0 and idd["status"] == 0, (im, idd)
    for um, ud in zip(Um, Ud):
        assert np.max(np.abs(um - ud)) / np.max(np.abs(ud)) < 1e-10


def test_batch_edge_sizes_and_validation(torch):
    import paper_2002_11978_gb300 as pkg
    M = 3
    inst, probs = _instances(torch, [(0, 31, 1.5, 0.5), (1, 33, 1.1, 0.7)], M)
    bs, U, info = _batch(torch, inst, M, precision="fp64")
    assert bs.shape[1] == 4  # n = 31 splits over at most 4 CTAs
    for p, u in zip(probs, U):
        ref, _ = _single(torch, p)
        assert np.max(np.abs(u - ref)) / np.max(np.abs(ref)) < 1e-10
    bad, _ = _instances(torch, [(0, 15, 1.5, 0.5)], M)
    with pytest.raises(pkg.TsfdeError) as e:
        pkg.BatchSolver(bad, M)
    assert e.value.status == pkg.TSFDE_ENOTSUP


def test_batch_partial_levels_and_cluster_sizes(torch):
    """Solving only the first K levels of the M-level mesh gives u^K of the
    single-problem march; every cluster size gives the same result."""
    import paper_2002_11978_gb300 as pkg
    M, K = 12, 5
    inst, probs = _instances(torch, [(20, 700, 1.4, 0.45), (21, 2100, 0.7, 0.6)], M)
    refs = []
    for p in probs:
        s = pkg.Solver(p.alpha, p.gamma, p.l, p.T, p.n, M, p.r, 1e-12)
        s.set_problem(cuda(torch, p.phi), cuda(torch, p.kappa0), None, None, F=[cuda(torch, p.F[0])],
                      G=[np.ones(M + 1)])
        u = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        for _ in range(K):
            s.step(u_out=u)
        refs.append(u.cpu().numpy())
    for q in (4, 8, 16):
        bs = pkg.BatchSolver(inst, M, precision="fp64", cluster_size=q)
        assert bs.shape[1] == q
        outs = [torch.zeros(d["n"], dtype=torch.float64, device="cuda") for d in inst]
        info = bs.solve(outs, levels=K)
        assert info["levels"] == 2 * K
        for u, ref in zip(outs, refs):
            assert np.max(np.abs(u.cpu().numpy() - ref)) / np.max(np.abs(ref)) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_warm_start_matches_cold(torch, precision):
    """Levels started from u^{m-1}, or from the extrapolated start, reach the
    cold-started FP64 solutions."""
    M = 24
    ns, al, ga = ti.batched_instance_params()
    specs = [(i, int(ns[i]), float(al[i]), float(ga[i])) for i in (3, 8, 64)]
    inst, probs = _instances(torch, specs, M)
    _, Uc, ic = _batch(torch, inst, M, precision="fp64")
    _, Uw, iw = _batch(torch, inst, M, precision=precision, warm_start=True)
    assert iw["status"] == 0, iw
    for a, b in zip(Uw, Uc):
        assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < 1e-10
    # the extrapolated start (warm_start = 2: the cubic in the level index
    # through u^{m-1} .. u^{m-4}) reaches the same solutions in fewer
    # iterations
    _, Ux, ix = _batch(torch, inst, M, precision=precision, warm_start="extrapolate")
    assert ix["status"] == 0, ix
    assert ix["iterations"] < iw["iterations"], (ix, iw)
    for a, b in zip(Ux, Uc):
        assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < 1e-10


def _mixed_specs():
    # sizes across both default size classes: two of the large one
    # (transforms of L = 16384 and 32768) and several small ones
    return [(0, 16383, 1.1, 0.3), (1, 9000, 1.5, 0.5), (2, 4000, 1.7, 0.8), (3, 2047, 0.7, 0.4),
            (4, 1500, 1.9, 0.6), (5, 700, 1.2, 0.2), (6, 511, 0.9, 0.9), (7, 3000, 1.4, 0.7)]


def test_batch_tuner_returns_the_fastest_plan_and_it_solves(torch):
    """tsfde_batch_tune times every launch plan that fits (one launch with
    cluster size 4, 8 or 16; two launches split at n = 8193 or 4097) on a
    probe solve and returns the fastest; a batch set up with that plan gives
    the default plan's u^M (mixed, warm start) to 1e-10."""
    import paper_2002_11978_gb300 as pkg
    M = 16
    inst, probs = _instances(torch, _mixed_specs(), M)
    best, tried = pkg.batch_tune(inst, M, probe_levels=2, precision="mixed", warm_start=True)
    assert len(tried) >= 2, tried
    assert best["probe_ms"] == min(t["probe_ms"] for t in tried), (best, tried)
    assert {t["classes"] for t in tried} == {1, 2}, tried
    _, U0, info0 = _batch(torch, inst, M, precision="mixed", warm_start=True)
    bs, U1, info1 = _batch(torch, inst, M, precision="mixed", warm_start=True, plan=best)
    got = bs.plan
    assert got["classes"] == best["classes"] and got["cluster_size"] == best["cluster_size"], (got, best)
    assert info0["status"] == 0 and info1["status"] == 0
    for a, b in zip(U0, U1):
        assert np.max(np.abs(a - b)) / np.max(np.abs(a)) < 1e-10


def test_batch_large_class_certified(torch):
    """Instances of the large size class (n >= 8193: transforms of L = 16384
    and 32768), mixed, warm start, on the batched workload's M = 1024 mesh.
    u^m for m = 1..8 comes from batched solves through level m (the launch
    is deterministic, so these are the levels of one march); at levels 2 and
    8 the residual certificate of the single-problem tests (oracle.certify:
    double-double defect with the direct FIDS history, Lemma 3.3) bounds the
    error by 1e-10 of max|u^m|.  The SOE table and the Toeplitz entries are
    the library's for the same parameters, read from a single-problem
    context (entries within two ulps of the oracle's)."""
    import math

    import paper_2002_11978_gb300 as pkg
    from oracle import certify
    M = 1024
    specs = [(0, 16383, 1.1, 0.3), (1, 9000, 1.5, 0.5), (2, 700, 1.7, 0.8)]
    inst, probs = _instances(torch, specs, M)
    bs = pkg.BatchSolver(inst, M, precision="mixed", warm_start=True)
    traj = [[p.phi.copy()] for p in probs]
    for m in range(1, 9):
        outs = [torch.zeros(d["n"], dtype=torch.float64, device="cuda") for d in inst]
        info = bs.solve(outs, levels=m)
        assert info["status"] == 0, info
        for k, u in enumerate(outs):
            traj[k].append(u.cpu().numpy())
    for k in (0, 1):
        p = probs[k]
        U = np.array(traj[k])
        ref = pkg.Solver(p.alpha, p.gamma, p.l, p.T, p.n, M, p.r, 1e-12)
        soe, t = ref.soe(), ref.symbol()  # the library's tables (see test_gpu_certificate.py)
        t_or = oracle.ifl_symbol(p.alpha, p.n)
        assert np.max(np.abs(t - t_or) / np.abs(t_or)) <= 5e-16  # two ulps
        for m in (2, 8):
            b = oracle.level_rhs("FIDS", p.alpha, p.gamma, p.l, p.T, p.r, p.n, M, m, U, p.F[0], soe=soe)
            ahat = oracle.l1_weight(p.T, M, p.r, p.gamma, m, m) / math.gamma(1 - p.gamma)
            bound, l33 = certify.certify_level(t, ahat, p.kappa0, U[m], b)
            assert bound <= 1e-10 * np.max(np.abs(U[m])), (p.n, m, bound, l33)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_pcg_matches_batch_bicgstab_at_workload_sizes(torch, precision):
    """The batched workload's size range (transforms of L = 1024 to 32768),
    M = 64 levels, warm start: PCG on the symmetrised system, the per-level
    choice (auto) and BiCGSTAB reach the same u^M (both stop at the same residual test; FP64 at 1e-13,
    as the benchmark compares the arms)."""
    M = 64
    inst, probs = _instances(torch, _mixed_specs(), M)
    tol = 1e-13 if precision == "fp64" else 1e-12
    _, Ub, ib = _batch(torch, inst, M, precision=precision, krylov="bicgstab", warm_start=True, krylov_tol=tol)
    for kry in ("pcg", "auto"):
        _, Up, ip = _batch(torch, inst, M, precision=precision, krylov=kry, warm_start=True, krylov_tol=tol)
        assert ib["status"] == 0 and ip["status"] == 0, (kry, ib, ip)
        for a, b in zip(Ub, Up):
            assert np.max(np.abs(a - b)) / np.max(np.abs(a)) < 1e-10, kry
