"""CPU-side checks of the C ABI: the library builds, loads without a GPU,
exports every entry point declared in include/tsfde.h, and rejects invalid
arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2002_11978_gb300 import build
    build.build()
    import paper_2002_11978_gb300 as pkg
    return pkg.load_library()


def declared_entry_points():
    text = open(os.path.join(ROOT, "include", "tsfde.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tsfde_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = declared_entry_points()
    assert "tsfde_setup" in names and "tsfde_step" in names and "tsfde_solve" in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_entry_points():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    import paper_2002_11978_gb300 as pkg
    assert sorted(pkg.exported_names()) == declared_entry_points()


def test_default_opts(lib):
    import paper_2002_11978_gb300 as pkg
    o = pkg.default_opts()
    assert o.krylov_tol == 1e-12 and o.precision == pkg.TSFDE_FP64 and o.max_it > 0


@pytest.mark.parametrize("args", [
    (0.0, 0.5, 1.0, 1.0, 7, 4, 3.0, 1e-12),    # alpha
    (2.0, 0.5, 1.0, 1.0, 7, 4, 3.0, 1e-12),
    (1.5, 0.0, 1.0, 1.0, 7, 4, 3.0, 1e-12),    # gamma
    (1.5, 1.0, 1.0, 1.0, 7, 4, 3.0, 1e-12),
    (1.5, 0.5, -1.0, 1.0, 7, 4, 3.0, 1e-12),   # l
    (1.5, 0.5, 1.0, 0.0, 7, 4, 3.0, 1e-12),    # T
    (1.5, 0.5, 1.0, 1.0, 0, 4, 3.0, 1e-12),    # n
    (1.5, 0.5, 1.0, 1.0, 7, 0, 3.0, 1e-12),    # M
    (1.5, 0.5, 1.0, 1.0, 7, 4, 0.5, 1e-12),    # r
    (1.5, 0.5, 1.0, 1.0, 7, 4, 3.0, 0.0),      # soe_tol
])
def test_setup_rejects_invalid_arguments(lib, args):
    import paper_2002_11978_gb300 as pkg
    ctx = ctypes.c_void_p()
    o = pkg.default_opts()
    rc = lib.tsfde_setup(ctypes.byref(ctx), *args, ctypes.byref(o))
    assert rc == pkg.TSFDE_EINVAL
    assert not ctx


def test_setup_rejects_bad_mu(lib):
    import paper_2002_11978_gb300 as pkg
    ctx = ctypes.c_void_p()
    o = pkg.default_opts()
    o.mu = 1.2  # must exceed alpha = 1.5
    assert lib.tsfde_setup(ctypes.byref(ctx), 1.5, 0.5, 1.0, 1.0, 7, 4, 3.0, 1e-12,
                           ctypes.byref(o)) == pkg.TSFDE_EINVAL


def test_null_context_calls_fail_cleanly(lib):
    import paper_2002_11978_gb300 as pkg
    assert lib.tsfde_reset(None) == pkg.TSFDE_EINVAL
    assert lib.tsfde_step(None, None, None, None, None, None) == pkg.TSFDE_EINVAL
    assert lib.tsfde_strerror(pkg.TSFDE_ETIMEOUT) == b"device barrier timed out"


def test_setup_rejects_unknown_engine(lib):
    import paper_2002_11978_gb300 as pkg
    ctx = ctypes.c_void_p()
    o = pkg.default_opts()
    assert o.engine == pkg.TSFDE_ENGINE_AUTO
    o.engine = 7
    assert lib.tsfde_setup(ctypes.byref(ctx), 1.5, 0.5, 1.0, 1.0, 7, 4, 3.0, 1e-12,
                           ctypes.byref(o)) == pkg.TSFDE_EINVAL
    assert not ctx
    assert lib.tsfde_get_engine(None) == -1


def test_setup_validates_history_and_precision(lib):
    import paper_2002_11978_gb300 as pkg
    ctx = ctypes.c_void_p()
    o = pkg.default_opts()
    assert o.history == pkg.TSFDE_HISTORY_SOE
    o.history = 5
    assert lib.tsfde_setup(ctypes.byref(ctx), 1.5, 0.5, 1.0, 1.0, 7, 4, 3.0, 1e-12,
                           ctypes.byref(o)) == pkg.TSFDE_EINVAL
    o = pkg.default_opts()
    o.precision = 3
    assert lib.tsfde_setup(ctypes.byref(ctx), 1.5, 0.5, 1.0, 1.0, 7, 4, 3.0, 1e-12,
                           ctypes.byref(o)) == pkg.TSFDE_EINVAL
    assert not ctx


def test_batch_rejects_direct_history(lib):
    """The batched solve is FIDS only: the direct history is refused before
    any device work."""
    import paper_2002_11978_gb300 as pkg
    o = pkg.default_opts()
    o.history = pkg.TSFDE_HISTORY_DIRECT
    inst = (pkg.tsfde_instance * 1)()
    inst[0] = pkg.tsfde_instance(1.5, 0.5, 1.0, 1.0, 3.0, 63, 1e-12, None, None, None)
    b = ctypes.c_void_p()
    assert lib.tsfde_batch_setup(ctypes.byref(b), 1, inst, 8, ctypes.byref(o)) == pkg.TSFDE_ENOTSUP
    assert not b


def test_setup_validates_krylov(lib):
    """An unknown method is refused, and PCG with the cluster engine (which
    runs BiCGSTAB only) is not supported; both before any device work."""
    import paper_2002_11978_gb300 as pkg
    ctx = ctypes.c_void_p()
    o = pkg.default_opts()
    assert o.krylov == pkg.TSFDE_KRYLOV_BICGSTAB
    o.krylov = 4
    assert lib.tsfde_setup(ctypes.byref(ctx), 1.5, 0.5, 1.0, 1.0, 7, 4, 3.0, 1e-12,
                           ctypes.byref(o)) == pkg.TSFDE_EINVAL
    o = pkg.default_opts()
    o.krylov = pkg.TSFDE_KRYLOV_PCG
    o.precision = pkg.TSFDE_MIXED
    o.engine = pkg.TSFDE_ENGINE_CLUSTER
    assert lib.tsfde_setup(ctypes.byref(ctx), 1.5, 0.5, 1.0, 1.0, 7, 4, 3.0, 1e-12,
                           ctypes.byref(o)) == pkg.TSFDE_ENOTSUP
    assert not ctx


def test_setup_validates_warm_start(lib):
    """warm_start takes 0 (x0 = 0), 1 (u^{m-1}) or 2 (extrapolated); other
    values are refused before any device work, single and batched."""
    import paper_2002_11978_gb300 as pkg
    ctx = ctypes.c_void_p()
    for w in (-1, 3):
        o = pkg.default_opts()
        o.warm_start = w
        assert lib.tsfde_setup(ctypes.byref(ctx), 1.5, 0.5, 1.0, 1.0, 7, 4, 3.0, 1e-12,
                               ctypes.byref(o)) == pkg.TSFDE_EINVAL
        inst = (pkg.tsfde_instance * 1)()
        inst[0] = pkg.tsfde_instance(1.5, 0.5, 1.0, 1.0, 3.0, 63, 1e-12, None, None, None)
        b = ctypes.c_void_p()
        assert lib.tsfde_batch_setup(ctypes.byref(b), 1, inst, 8, ctypes.byref(o)) == pkg.TSFDE_EINVAL
        assert not b
    assert not ctx
    assert pkg._warm("extrapolate") == 2 and pkg._warm(True) == 1 and pkg._warm(False) == 0


def test_batch_krylov_option(lib):
    """The batched solve accepts BiCGSTAB, PCG and AUTO, and rejects other
    values; an instance with NULL data pointers is rejected before any
    device work."""
    import paper_2002_11978_gb300 as pkg
    o = pkg.default_opts()
    inst = (pkg.tsfde_instance * 1)()
    inst[0] = pkg.tsfde_instance(1.5, 0.5, 1.0, 1.0, 3.0, 63, 1e-12, None, None, None)
    b = ctypes.c_void_p()
    o.krylov = 7
    assert lib.tsfde_batch_setup(ctypes.byref(b), 1, inst, 8, ctypes.byref(o)) == pkg.TSFDE_EINVAL
    for k in (pkg.TSFDE_KRYLOV_PCG, pkg.TSFDE_KRYLOV_AUTO):
        o.krylov = k
        assert lib.tsfde_batch_setup(ctypes.byref(b), 1, inst, 8, ctypes.byref(o)) == pkg.TSFDE_EINVAL
    assert not b
