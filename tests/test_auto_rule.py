"""The per-level Krylov choice rule (auto_rule_next in csrc/plan.h), compiled
for the host and driven with scripted level times.

The rule is host-and-device code; the GPU kernels run the same function
(levels.cuh for the grid engine, batch.cu for the batched engine).  Here a
small host program feeds it the device time of each level for the method
that ran, and the test reads back which method every level took.  The
expected positions follow from the rule's statement: level 1 BiCGSTAB,
level 2 a trial of PCG, then a trial of the slower method 8 r^2 levels
(8..64) after its latest sample, doubled per trial of it lost in a row."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2002_11978_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

HARNESS = r"""
#include <cstdio>
#include "plan.h"
int main() {
  tsfde::AutoRule k;
  tsfde::auto_rule_init(k);
  int me = 0;
  long long m = 0;
  double tb, tp;
  while (std::scanf("%lf %lf", &tb, &tp) == 2) {
    ++m;
    std::printf("%d", me);
    me = tsfde::auto_rule_next(k, me, m, me ? tp : tb);
  }
  std::printf("\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def rule(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("auto_rule")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(HARNESS)
    subprocess.check_call([cxx, "-std=c++17", "-O1", f"-I{CUDA_INC}", f"-I{CSRC}", str(src), "-o", str(exe)])

    def run(times):
        """times: list of (BiCGSTAB ms, PCG ms) per level; returns the
        method string, one character per level ('0' BiCGSTAB, '1' PCG)."""
        inp = "".join(f"{a!r} {b!r}\n" for a, b in times)
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout
        return out.strip()

    return run


def switches(s):
    """1-based levels whose method differs from the previous level's."""
    return [i + 1 for i in range(1, len(s)) if s[i] != s[i - 1]]


def test_slower_pcg_is_retried_at_doubling_intervals(rule):
    # PCG twice as slow throughout: r = 2, 8 r^2 = 32 levels, doubled per lost trial
    s = rule([(1.0, 2.0)] * 400)
    assert s[0] == "0" and s[1] == "1"          # level 1 BiCGSTAB, level 2 the first trial
    # trials at 2 (lost: next after 64 levels), 66 (lost: 128), 194 (lost: 256 ... capped at 16x)
    assert switches(s) == [2, 3, 66, 67, 194, 195]
    assert s.count("1") == 3


def test_faster_pcg_keeps_the_march(rule):
    # PCG twice as fast: the march stays with it; BiCGSTAB's trials lose
    s = rule([(2.0, 1.0)] * 200)
    assert switches(s) == [2, 33, 34, 97, 98]   # BiCGSTAB trials at 33 (32 after level 1) and 97
    assert s.count("0") == 3


def test_crossover_is_followed(rule):
    # BiCGSTAB faster for 100 levels, PCG faster after: the march moves to
    # PCG at its next trial and stays; the extra time stays small
    times = [(1.0, 1.5)] * 100 + [(1.5, 1.0)] * 300
    s = rule(times)
    cross = [i + 1 for i in range(100, 400) if s[i] == "1"]
    assert cross and cross[0] <= 101 + 64 * 16
    assert s[cross[0]:].count("0") <= 4         # a few BiCGSTAB trials after the switch
    spent = sum(t[int(c)] for t, c in zip(times, s))
    best = sum(min(t) for t in times)
    assert spent <= 1.5 * best


def test_failed_level_switches_method(rule):
    # a failed PCG level (infinitely slow) sends the march back to BiCGSTAB,
    # and a failed BiCGSTAB level sends it to PCG, trial or not
    inf = float("inf")
    s = rule([(1.0, 1.0), (1.0, inf), (1.0, 1.0), (1.0, 1.0)])
    assert s[:3] == "010"
    s = rule([(1.0, 2.0), (1.0, 2.0), (inf, 2.0), (1.0, 2.0)])
    assert s[:4] == "0101"


def test_equal_times_do_not_oscillate(rule):
    # a tie counts as a win for the method that ran, so the march changes
    # method only when a trial is due (every 8 levels at r = 1), never on
    # consecutive levels
    s = rule([(1.0, 1.0)] * 100)
    sw = switches(s)
    assert all(b - a >= 7 for a, b in zip(sw[1:], sw[2:]))
