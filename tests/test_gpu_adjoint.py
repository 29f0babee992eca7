"""GPU adjoint sweep (tsfde_adjoint): the transposed FP64 level solves with
the reversed SOE recurrence, against the oracle's dense adjoint (direct FIDS
weights, dense transposed LU), against central differences of J through the
GPU forward march, through torch.autograd, and at the full adjoint workload
size (n = 4095, M = 1024)."""
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


def _setup(torch, n, M, soe=None, **kw):
    import paper_2002_11978_gb300 as pkg
    prob, kobs = ti.config_adjoint(n=n, M=M)
    s = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, n, M, prob.r, 1e-12, soe=soe, **kw)
    return pkg, prob, kobs, s


def _forward(torch, s, prob, kap, f):
    s.set_problem(cuda(torch, prob.phi), cuda(torch, kap), None, None, F=[cuda(torch, f)],
                  G=[np.ones(prob.M + 1)])
    U = torch.zeros((prob.M + 1, prob.n), dtype=torch.float64, device="cuda")
    uf = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    info = s.solve(uf, U)
    assert info["status"] == 0, info
    return U


@pytest.mark.parametrize("n,M,krylov", [(255, 32, "bicgstab"), (63, 16, "bicgstab"), (1, 4, "bicgstab"),
                                        (7, 1, "bicgstab"), (255, 32, "pcg"), (63, 16, "pcg"),
                                        (1, 4, "pcg"), (255, 32, "auto")])
def test_adjoint_matches_dense_oracle(torch, n, M, krylov):
    """Same SOE table on both sides; the oracle solves every transposed level
    system by dense LU with the direct FIDS weights.  Forward and transposed
    solves run to a relative residual of 1e-14: the gradient is within about
    cond(level matrix) x tol of the dense one (cond ~1e3-1e4 at n = 255),
    so 1e-14 is what brings it under 1e-10.  The transposed solves run
    BiCGSTAB, or PCG on (ahat K^{-1} + A) mu = g with lambda = K^{-1} mu, or
    (auto) the method the forward march chose at each level."""
    prob, kobs = ti.config_adjoint(n=n, M=M)
    tm, tau = oracle.graded_mesh(prob.T, M, prob.r)
    soe = oracle.soe_build(prob.gamma, tau[1], prob.T, 1e-12)
    _, _, _, s = _setup(torch, n, M, soe=soe, krylov_tol=1e-14, krylov=krylov)
    f0 = prob.F[0]
    u_obs = oracle.march("FIDS", prob.alpha, prob.gamma, prob.l, prob.T, prob.r, n, M, prob.phi,
                         np.tile(kobs, (M + 1, 1)), np.tile(f0, (M + 1, 1)), soe=soe)[M]
    J0, Uo, gk_ref, gf_ref = oracle.adjoint(prob.alpha, prob.gamma, prob.l, prob.T, prob.r, n, M,
                                            prob.phi, prob.kappa0, f0, u_obs, soe)
    U = _forward(torch, s, prob, prob.kappa0, f0)
    assert np.max(np.abs(U.cpu().numpy() - Uo)) / np.max(np.abs(Uo)) < 1e-10
    gk = torch.zeros(n, dtype=torch.float64, device="cuda")
    gf = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = s.adjoint(U, U[M] - cuda(torch, u_obs), gk, gf)
    assert info["status"] == 0 and info["iterations"] > 0, info
    ek = np.max(np.abs(gk.cpu().numpy() - gk_ref)) / np.max(np.abs(gk_ref))
    ef = np.max(np.abs(gf.cpu().numpy() - gf_ref)) / np.max(np.abs(gf_ref))
    assert ek < 1e-10 and ef < 1e-10, (ek, ef, info)


@pytest.mark.parametrize("stride,kw", [(6, {}), (-1, {}), (1, {}), (32, {}),
                                       (6, dict(warm_start="extrapolate", krylov="auto")),
                                       (1, dict(warm_start="extrapolate", krylov="auto"))])
def test_checkpointed_adjoint_equals_trajectory_adjoint(torch, stride, kw):
    """u_all = NULL: the sweep marches each segment between checkpoints again
    (stride 6 leaves a ragged last segment of 2 levels at M = 32; -1 is
    ceil(sqrt(M)) = 6; 1 and M are the extremes).  The recomputed levels run
    the same deterministic kernels from the same state (with an extrapolated
    start, the checkpoint's three levels feed it; with the per-level Krylov
    choice, the method the forward march recorded for the level), so the
    gradients equal those of the sweep over the stored trajectory, and the
    forward state is left where it was."""
    n, M = 255, 32
    _, prob, kobs, s = _setup(torch, n, M, ckpt_stride=stride, **kw)
    f0 = prob.F[0]
    u_obs = _forward(torch, s, prob, kobs, f0)[M].clone()
    U = _forward(torch, s, prob, prob.kappa0, f0)
    g = {}
    for mode in ("trajectory", "checkpoints"):
        gk = torch.zeros(n, dtype=torch.float64, device="cuda")
        gf = torch.zeros(n, dtype=torch.float64, device="cuda")
        info = s.adjoint(U if mode == "trajectory" else None, U[M] - u_obs, gk, gf)
        assert info["status"] == 0, info
        assert info["recomputed_levels"] == (M if mode == "checkpoints" else 0), info
        g[mode] = (gk.cpu().numpy(), gf.cpu().numpy())
    for a, b in zip(g["trajectory"], g["checkpoints"]):
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a)), np.max(np.abs(a - b))
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.current_solution(u)
    assert torch.equal(u, U[M])


def test_checkpointed_adjoint_needs_a_whole_march(torch):
    import paper_2002_11978_gb300 as pkg
    n, M = 63, 8
    _, prob, kobs, s = _setup(torch, n, M, ckpt_stride=-1)
    s.set_problem(cuda(torch, prob.phi), cuda(torch, prob.kappa0), None, None,
                  F=[cuda(torch, prob.F[0])], G=[np.ones(M + 1)])
    s.step()
    gk = torch.zeros(n, dtype=torch.float64, device="cuda")
    gf = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.TsfdeError) as e:
        s.adjoint(None, gk.clone(), gk, gf)
    assert e.value.status == pkg.TSFDE_ESTATE
    s2 = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, n, M, prob.r, 1e-12)
    s2.set_problem(cuda(torch, prob.phi), cuda(torch, prob.kappa0))
    s2.solve(torch.zeros(n, dtype=torch.float64, device="cuda"))
    with pytest.raises(pkg.TsfdeError) as e:
        s2.adjoint(None, gk.clone(), gk, gf)
    assert e.value.status == pkg.TSFDE_ESTATE


def test_adjoint_vs_central_differences_on_gpu(torch):
    n, M = 1023, 64
    _, prob, kobs, s = _setup(torch, n, M)
    f0 = prob.F[0]
    u_obs = _forward(torch, s, prob, kobs, f0)[M].clone()

    def J(kap, f):
        U = _forward(torch, s, prob, kap, f)
        return 0.5 * float(torch.sum((U[M] - u_obs) ** 2))

    U = _forward(torch, s, prob, prob.kappa0, f0)
    gk = torch.zeros(n, dtype=torch.float64, device="cuda")
    gf = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.adjoint(U, U[M] - u_obs, gk, gf)
    gk, gf = gk.cpu().numpy(), gf.cpu().numpy()
    rng = np.random.default_rng(3)
    for _ in range(2):
        d = rng.standard_normal(n)
        d /= np.linalg.norm(d)
        hk = 1e-5 * np.max(prob.kappa0)
        fd_k = (J(prob.kappa0 + hk * d, f0) - J(prob.kappa0 - hk * d, f0)) / (2 * hk)
        fd_f = (J(prob.kappa0, f0 + 1e-5 * d) - J(prob.kappa0, f0 - 1e-5 * d)) / 2e-5
        assert gk @ d == pytest.approx(fd_k, rel=1e-5), (gk @ d, fd_k)
        assert gf @ d == pytest.approx(fd_f, rel=1e-5), (gf @ d, fd_f)


@pytest.mark.parametrize("stride", [0, -1])
def test_autograd_function_matches_oracle(torch, stride):
    """Through torch.autograd, with the trajectory kept (stride 0) or with
    checkpoints (-1: the backward pass marches the segments again)."""
    from paper_2002_11978_gb300.autograd import fids_solve
    n, M = 255, 24
    prob, kobs = ti.config_adjoint(n=n, M=M)
    tm, tau = oracle.graded_mesh(prob.T, M, prob.r)
    soe = oracle.soe_build(prob.gamma, tau[1], prob.T, 1e-12)
    _, _, _, s = _setup(torch, n, M, soe=soe, krylov_tol=1e-14, ckpt_stride=stride)
    f0 = prob.F[0]
    u_obs = oracle.march("FIDS", prob.alpha, prob.gamma, prob.l, prob.T, prob.r, n, M, prob.phi,
                         np.tile(kobs, (M + 1, 1)), np.tile(f0, (M + 1, 1)), soe=soe)[M]
    _, _, gk_ref, gf_ref = oracle.adjoint(prob.alpha, prob.gamma, prob.l, prob.T, prob.r, n, M,
                                          prob.phi, prob.kappa0, f0, u_obs, soe)
    kap = cuda(torch, prob.kappa0).requires_grad_(True)
    f = cuda(torch, f0).requires_grad_(True)
    uM = fids_solve(kap, f, s, cuda(torch, prob.phi))
    J = 0.5 * torch.sum((uM - cuda(torch, u_obs)) ** 2)
    J.backward()
    assert np.max(np.abs(kap.grad.cpu().numpy() - gk_ref)) / np.max(np.abs(gk_ref)) < 1e-10
    assert np.max(np.abs(f.grad.cpu().numpy() - gf_ref)) / np.max(np.abs(gf_ref)) < 1e-10


def test_adjoint_keeps_forward_state(torch):
    """An adjoint call between forward steps leaves the march where it was."""
    n, M = 127, 8
    _, prob, kobs, s = _setup(torch, n, M)
    f0 = prob.F[0]
    U = _forward(torch, s, prob, prob.kappa0, f0)
    s.set_problem(cuda(torch, prob.phi), cuda(torch, prob.kappa0), None, None,
                  F=[cuda(torch, f0)], G=[np.ones(M + 1)])
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    for _ in range(3):
        s.step(u_out=u)
    gk = torch.zeros(n, dtype=torch.float64, device="cuda")
    gf = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.adjoint(U, U[M].clone(), gk, gf)
    for m in range(4, M + 1):
        s.step(u_out=u)
    assert torch.equal(u, U[M])


def test_adjoint_rejects_time_dependent_kappa(torch):
    import paper_2002_11978_gb300 as pkg
    n, M = 31, 4
    s = pkg.Solver(1.4, 0.5, 1.0, 1.0, n, M, 3.0, 1e-12)
    one = torch.ones(n, dtype=torch.float64, device="cuda")
    s.set_problem(one, one, one, np.ones(M + 1))
    U = torch.zeros((M + 1, n), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.TsfdeError) as e:
        s.adjoint(U, one, one.clone(), one.clone())
    assert e.value.status == pkg.TSFDE_ENOTSUP


def test_adjoint_full_workload_size_20_directions(torch):
    """The adjoint workload, n = 4095, M = 1024, with sqrt(M) checkpointing
    (u_all = NULL): every transposed level converges, and along 20 seeded
    random directions (d_kappa, d_f) the gradient matches a central
    difference of J(t) = J(kappa + t s_k d_kappa, f + t s_f d_f) with
    h = 1e-6 (s_k = max kappa, s_f = max |f|) through the GPU forward march,
    forward and adjoint solves at 1e-14, to 1e-6 relative."""
    import paper_2002_11978_gb300 as pkg
    n, M = 4095, 1024
    prob, kobs = ti.config_adjoint(n=n, M=M)
    s = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, n, M, prob.r, 1e-12, krylov_tol=1e-14,
                   ckpt_stride=-1)
    f0 = prob.F[0]
    uf = torch.zeros(n, dtype=torch.float64, device="cuda")

    def uM(kap, f):
        s.set_problem(cuda(torch, prob.phi), cuda(torch, kap), None, None, F=[cuda(torch, f)],
                      G=[np.ones(M + 1)])
        info = s.solve(uf)
        assert info["status"] == 0, info
        return uf.clone()

    u_obs = uM(kobs, f0)
    u = uM(prob.kappa0, f0)
    gk = torch.zeros(n, dtype=torch.float64, device="cuda")
    gf = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = s.adjoint(None, u - u_obs, gk, gf)
    assert info["status"] == 0 and info["recomputed_levels"] == M, info
    gk, gf = gk.cpu().numpy(), gf.cpu().numpy()
    J = lambda kap, f: 0.5 * float(torch.sum((uM(kap, f) - u_obs) ** 2))
    sk, sf, h = float(np.max(prob.kappa0)), float(np.max(np.abs(f0))), 1e-6
    rng = np.random.default_rng(20)
    worst = 0.0
    for _ in range(20):
        dk = rng.standard_normal(n)
        df = rng.standard_normal(n)
        dk /= np.linalg.norm(dk)
        df /= np.linalg.norm(df)
        fd = (J(prob.kappa0 + h * sk * dk, f0 + h * sf * df) -
              J(prob.kappa0 - h * sk * dk, f0 - h * sf * df)) / (2 * h)
        ad = sk * (gk @ dk) + sf * (gf @ df)
        worst = max(worst, abs(ad - fd) / abs(fd))
    assert worst < 1e-6, worst
