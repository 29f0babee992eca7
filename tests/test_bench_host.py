"""Host logic of bench.py that needs no GPU: the digest that keys the
recorded DRAM traffic figure to the kernel code it was measured on.

The figure must survive an edit of comments or spacing in the kernel
sources (the compiled kernels are the same) and must disappear (null in the
bench line) once the code itself changes."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_recorded_traffic_matches_the_current_kernel_code(bench):
    for kernel, rec in bench.TRAFFIC.items():
        assert bench.measured_traffic(kernel) == rec["bytes"], (
            kernel, "kernel code changed since the traffic capture; capture it again")


def test_digest_ignores_comments_and_spacing_but_not_code(bench, tmp_path, monkeypatch):
    src = tmp_path / "paper_2002_11978_gb300" / "csrc"
    src.mkdir(parents=True)
    code = "// header\nint f(int x) {\n  return x + 1;  // one\n}\n/* block\n comment */\n"
    (src / "a.cu").write_text(code)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.code_digest(["a.cu"])
    (src / "a.cu").write_text("// another header\nint f(int x)\n{\n    return x + 1;\n}\n")
    assert bench.code_digest(["a.cu"]) == d0
    (src / "a.cu").write_text(code.replace("x + 1", "x + 2"))
    assert bench.code_digest(["a.cu"]) != d0
    # and the real sources' digest is what the record holds
    monkeypatch.setattr(bench, "ROOT", ROOT)
    for rec in bench.TRAFFIC.values():
        assert bench.code_digest(rec["sources"]) == rec["sha1"]
