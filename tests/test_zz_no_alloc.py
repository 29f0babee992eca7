"""The allocation-free Toeplitz product (tsfde_toeplitz_apply_static).

Some callers cannot call cudaMalloc: code whose device memory all comes from
a framework's pool, or a thread that must not trigger the allocator's
implicit synchronisation.  For them the library offers y = A v with every
work buffer in one fixed array inside the library, reused by every call.
Two calls in a row must each give the same product as the oracle's direct
O(n^2) sum and as the context-based tsfde_toeplitz_apply built with the same
splitting.  This file is collected last, so a stop-at-first-failure run has
already run every other test."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2002_11978_gb300 import build
    build.build()
    return T


def _tol(n):
    # the bound tests/test_gpu_parity.py puts on an FP64 Toeplitz product, per
    # unit of ||A||_inf ||v||_inf
    L = max(8, 1 << math.ceil(math.log2(max(2 * n - 1, 1))))
    return 4e-16 * math.log2(L) * 4


# (alpha, mu, kappa_mu, l): the default splitting mu = 1 + alpha/2 with
# kappa_mu = 1, the paper's other choice mu = 2 with kappa_mu = 2, another
# mu with kappa_mu = 1, and a half-width l != 1
SPLITS = [(1.5, None, None, 1.0), (1.5, 2.0, 2, 1.0), (1.2, 1.9, 1, 1.0), (0.7, None, None, 2.5)]


@pytest.mark.parametrize("n", [1, 7, 127, 1000, 16383])
@pytest.mark.parametrize("alpha,mu,kmu,l", SPLITS)
def test_static_product_matches_oracle_and_context_on_two_calls(torch, n, alpha, mu, kmu, l):
    import paper_2002_11978_gb300 as pkg
    t = oracle.ifl_symbol(alpha, n, l=l, mu=mu, kappa_mu=kmu)
    s = pkg.Solver(alpha, 0.5, l, 1.0, n, 4, 3.0, 1e-12, mu=mu, kappa_mu=kmu)
    scale = t[0] + 2 * np.sum(np.abs(t[1:]))
    rng = np.random.default_rng(n)
    for call in range(2):
        v_h = rng.standard_normal(n)
        v = torch.as_tensor(v_h, dtype=torch.float64, device="cuda")
        y_ctx = torch.zeros(n, dtype=torch.float64, device="cuda")
        y = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        s.toeplitz_apply(v, y_ctx, "fp64")
        pkg.toeplitz_apply_static(alpha, n, v, y, l=l, mu=mu, kappa_mu=kmu)
        ref = oracle.toeplitz_matvec(t, v_h)
        norm = scale * np.max(np.abs(v_h))
        err_orc = np.max(np.abs(y.cpu().numpy() - ref)) / norm
        err_ctx = float(torch.max(torch.abs(y - y_ctx))) / norm
        assert err_orc < _tol(n), (call, err_orc)
        assert err_ctx < _tol(n), (call, err_ctx)


def test_static_product_rejects_n_beyond_capacity(torch):
    import paper_2002_11978_gb300 as pkg
    n = 16384
    v = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.TsfdeError) as e:
        pkg.toeplitz_apply_static(1.5, n, v, y)
    assert e.value.status == pkg.TSFDE_ENOTSUP
