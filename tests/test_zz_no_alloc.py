"""The allocation-free Toeplitz product (tsfde_toeplitz_apply_static) must
give the same y = A v as the context-based tsfde_toeplitz_apply, call after
call, although all of its work buffers live in one fixed array that every
call reuses.  Callers that cannot allocate device memory use it; this file
is collected last so a stop-at-first-failure run has already run the rest."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2002_11978_gb300 import build
    build.build()
    return T


def _tol(n):
    # the bound tests/test_gpu_parity.py puts on a Toeplitz product, per unit
    # of ||A||_inf ||v||_inf
    L = max(8, 1 << math.ceil(math.log2(max(2 * n - 1, 1))))
    return 4e-16 * math.log2(L) * 4


@pytest.mark.parametrize("n,alpha", [(1, 1.5), (7, 0.5), (127, 1.5), (1000, 1.9), (16383, 1.6)])
def test_static_product_matches_context_product_on_two_calls(torch, n, alpha):
    import paper_2002_11978_gb300 as pkg
    s = pkg.Solver(alpha, 0.5, 1.0, 1.0, n, 4, 3.0, 1e-12)
    t = s.symbol()
    scale = t[0] + 2 * np.sum(np.abs(t[1:]))
    rng = np.random.default_rng(n)
    for call in range(2):
        v = torch.as_tensor(rng.standard_normal(n), dtype=torch.float64, device="cuda")
        y_ref = torch.zeros(n, dtype=torch.float64, device="cuda")
        y = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        s.toeplitz_apply(v, y_ref, "fp64")
        pkg.toeplitz_apply_static(alpha, n, v, y)
        err = float(torch.max(torch.abs(y - y_ref))) / (scale * float(torch.max(torch.abs(v))))
        assert err < _tol(n), (call, err)


def test_static_product_rejects_n_beyond_capacity(torch):
    import paper_2002_11978_gb300 as pkg
    n = 16384
    v = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.TsfdeError) as e:
        pkg.toeplitz_apply_static(1.5, n, v, y)
    assert e.value.status == pkg.TSFDE_ENOTSUP
