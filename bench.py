#!/usr/bin/env python3
"""Benchmark of the FIDS hot path on the headline workload:
n = 2^17 - 1 interior points, M = 4096 graded levels, gamma = 0.4 (r = 4),
alpha = 1.6, kappa = exp(GRF) mapped onto [0.2, 5], mixed precision
(double-single inner PBiCGSTAB inside FP64 refinement; --inner fp32 for the
FP32 inner solver) vs the plain FP64 path.

One step = one time level of the scheme: SOE history update and
right-hand side, Strang preconditioner for the level, Krylov solve (from
the cubic extrapolation 4 u^{m-1} - 6 u^{m-2} + 4 u^{m-3} - u^{m-4}, stopping at
||r|| < 1e-12 ||b||; --start prev: from u^{m-1}; --cold-start: from x0 = 0,
the paper's setting, with the same stopping rule).  A `batched` object adds the
512-problem workload (first 128 of its 1024 levels), an `adjoint` object the
gradient sweep of the adjoint workload (n = 4095, M = 1024).
Steps are timed one by one with CUDA events on the solver's stream; L2 is
flushed (256 MB write, then a 256 MB read so that no dirty flush lines are
left to write back) outside the events before every timed level.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).  Under torchrun each rank runs an independent
replica on its own GPU (a single problem does not shard: its levels are
sequential); value = levels of all ranks / max elapsed.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "steps/s & % HBM roofline at N=2^17-1, M=4096: mixed vs FP64, rel err <=1e-10"
WORKLOAD = "fids-mixed n=131071 M=4096 gamma=0.4 r=4 alpha=1.6 kappa=GRF[0.2,5]"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed levels (default: rest of the march)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=131071)
    ap.add_argument("--M", type=int, default=4096)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison arm")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-n", type=int, default=2047)
    ap.add_argument("--start", choices=["extrapolate", "prev", "zero"], default="extrapolate",
                    help="initial guess of each level solve: cubic extrapolation in the level "
                         "index (default), u^{m-1}, or 0; same stopping rule ||r|| < tol ||b||")
    ap.add_argument("--cold-start", action="store_true",
                    help="x0 = 0 for every level as in the paper's experiments (= --start zero)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint workload")
    ap.add_argument("--no-mid", action="store_true", help="skip the mid workload (n = 2^14 - 1, six pairs)")
    ap.add_argument("--dids-levels", type=int, default=None,
                    help="levels of the DIDS (direct history) march to time; default M, 0 skips it")
    ap.add_argument("--krylov", choices=["auto", "bicgstab", "pcg"], default="auto",
                    help="level solver of the mixed and FP64 arms: per-level choice between PCG on the "
                         "symmetrised system and BiCGSTAB from measured level times (auto), or one of "
                         "them throughout; unless bicgstab, the paper's FP64 BiCGSTAB is reported too")
    ap.add_argument("--flush-mb", type=int, default=256,
                    help="L2 flush buffer size (MB, twice L2 by default); smaller only for profiler runs")
    ap.add_argument("--inner", choices=["fp32", "ds"], default="ds",
                    help="arithmetic of the mixed arm's inner PBiCGSTAB: FP32, or double-single "
                         "(FP32 pairs, ~48-bit significand)")
    ap.add_argument("--batched-levels", type=int, default=128,
                    help="levels of the batched workload on which mixed and FP64 are compared (of "
                         "M = 1024; 0 skips the batched workload)")
    ap.add_argument("--no-batched-full", action="store_true",
                    help="skip timing the batched mixed path over all M = 1024 levels")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def shard(count, rank, world):
    """Instances of a batched workload on this rank: i with i mod world == rank
    (independent problems, no exchange between ranks)."""
    return [i for i in range(count) if i % world == rank]


def max_over_ranks(values, device):
    """Element-wise maximum of per-rank times over all ranks (the job's wall
    time is the slowest rank's)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# working set of the L2 probe: the level solve's resident vectors and FFT
# buffers at n = 2^17 - 1 take a few tens of MB
L2_PROBE_MB = 48


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def measured_l2_peak(torch, pkg, stream, mb=L2_PROBE_MB, reps=64, trials=5):
    """L2 read bandwidth in GB/s: tsfde_probe_l2_read over an mb-MB buffer
    (resident in L2 after one untimed pass), the best of `trials` timed
    passes of `reps` sweeps each, CUDA events on the probe's stream."""
    buf = torch.ones(mb * 2 ** 20 // 8, dtype=torch.float64, device="cuda")
    best = 0.0
    with torch.cuda.stream(stream):
        pkg.probe_l2_read(buf, 1, stream)
        for _ in range(trials):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pkg.probe_l2_read(buf, reps, stream)
            e1.record(stream)
            e1.synchronize()
            best = max(best, buf.numel() * 8.0 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    del buf
    return best


# ---------------------------------------------------------------- our arm
# DRAM bytes per level of the double-single level kernels from one ncu capture
# (profiles/k_level_mixed_ds_n131071_launches_traffic.md), valid only for the code
# they were taken with: the digest of that code (code_digest: comments and blank
# space ignored) is kept beside the figure, and changed code makes the figure null.
TRAFFIC = {"k_level_mixed_ds/auto": {
    "bytes": 62.8e6,
    "note": "dram read+write per level (k_precond_ds and both method kernels) at levels 6-11, ncu; "
            "BiCGSTAB levels of 8-11 inner iterations; the PCG levels of the late march take ~5",
    "sources": ['grid.cuh', 'levels.cuh', 'levelds.cu', 'levelds_pcg.cu', 'dev.cuh', 'dsf.cuh',
                'plan.h', 'abi.cpp', 'kernels.cu'],
    "sha1": "7b041ade0cfad06dd955660ce2f1bd65778f049d"}}


def code_digest(files):
    """SHA-1 of the code of the given csrc files with comments and blank
    space removed: a change of code changes it, a change of comments does not."""
    import hashlib
    import re
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_2002_11978_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()


def measured_traffic(kernel):
    t = TRAFFIC.get(kernel)
    if t is None:
        return None
    return t["bytes"] if code_digest(t["sources"]) == t["sha1"] else None


def run_arm(torch, pkg, prob, precision, W, K, flush, stream, e2e=False, warm=False, krylov="bicgstab"):
    """March W untimed levels, then K timed levels (restarting the march
    after level M).  Each timed level is bracketed by CUDA events on the
    solver's stream, with an L2 flush before it.  Returns the solver, the
    per-level milliseconds, the per-kernel event totals and the iteration
    totals of the timed levels."""
    s = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, prob.n, prob.M, prob.r, prob.soe_tol,
                   precision=precision, krylov_tol=1e-12, profile=True, stream=stream,
                   warm_start=warm, krylov=krylov)
    s.set_problem_from(prob)
    n = prob.n
    dev = torch.device("cuda")
    tot = {"its": 0, "outer": 0, "E_active_sum": 0, "status": 0, "fallback": 0, "max_relres": 0.0,
           "above_tol": 0, "its_pcg": 0, "levels_pcg": 0, "levels": 0}
    if e2e:
        kap_h = torch.from_numpy(prob.kappa0.copy()).pin_memory()
        f_h = torch.from_numpy(prob.f_at(0.0)).pin_memory()
        u_h = torch.empty(n, dtype=torch.float64).pin_memory()
        kap_d = torch.empty(n, dtype=torch.float64, device=dev)
        f_d = torch.empty(n, dtype=torch.float64, device=dev)
        u_d = torch.empty(n, dtype=torch.float64, device=dev)
    first_timed = [None]

    def collect():
        if first_timed[0] is not None and s.m >= first_timed[0]:
            for rec in s.level_stats(first_timed[0], s.m):
                tot["its"] += rec["iterations"]
                tot["levels"] += 1
                if rec["krylov"] == 1:
                    tot["its_pcg"] += rec["iterations"]
                    tot["levels_pcg"] += 1
                tot["outer"] += abs(rec["outer"])  # negative: finished by the FP64 fallback
                tot["fallback"] += rec["outer"] < 0
                tot["E_active_sum"] += rec["E_active"]
                tot["status"] = tot["status"] or rec["status"]
                tot["max_relres"] = max(tot["max_relres"], rec["rel_residual"])
                tot["above_tol"] += rec["rel_residual"] > 1e-12

    def one_level(timed):
        if s.m == prob.M:
            collect()
            s.reset()
            if timed:
                first_timed[0] = 1
        if timed and first_timed[0] is None:
            first_timed[0] = s.m + 1
        if e2e:
            kap_d.copy_(kap_h, non_blocking=True)
            f_d.copy_(f_h, non_blocking=True)
            s.step(kappa_m=kap_d, f_m=f_d, u_out=u_d, sync=False)
            u_h.copy_(u_d, non_blocking=True)
        else:
            s.step(sync=False)

    with torch.cuda.stream(stream):
        for _ in range(W):
            one_level(False)
        torch.cuda.synchronize()
        s.timing()  # discard the warm-up kernel times
        evs = []
        for _ in range(K):
            flush[0].zero_()            # write a buffer larger than L2 ...
            flush[1].sum(dtype=torch.float64)  # ... then read another, so that the
            # level does not start by writing the flush's dirty lines back to HBM
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_level(True)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    tim = s.timing()
    collect()
    return s, ms, tim, tot


def batched_sample(torch, pkg, ti, levels, rank, world, stream, warm=True, full=True):
    """The batched workload: 512 independent problems (n log-uniform in
    [2^9-1, 2^14-1], alpha ~ U(0.6, 1.9), gamma ~ U(0.2, 0.9), M = 1024),
    this rank's share (instance i on rank i mod world).  The launch plan
    (one persistent launch or two size classes, cluster size per launch) is
    chosen by tsfde_batch_tune on a 4-level probe and reported with every
    plan it timed.  Timed with CUDA events, with the per-level choice of
    BiCGSTAB or PCG inside each instance's march: mixed and FP64 over the
    first `levels` levels, the paper's FP64 BiCGSTAB on the same levels, and
    the mixed path over all M levels (full=True).  Its working set (the SOE
    histories, ~3 GB) is far above L2."""
    M = 1024
    ns, al, ga = ti.batched_instance_params()
    mine = shard(len(ns), rank, world)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    inst = []
    for i in mine:
        p = ti.config_batched_instance(i, int(ns[i]), float(al[i]), float(ga[i]), M=M)
        inst.append(dict(alpha=p.alpha, gamma=p.gamma, n=p.n, r=p.r, phi=dev(p.phi),
                         kappa=dev(p.kappa0), f=dev(p.F[0])))
    unknowns = sum(d["n"] for d in inst)
    out = {"workload": "fids-batched 512 instances n=U_log[511,16383] M=1024 (alpha, gamma random)",
           "instances": len(inst), "levels_compared": levels, "unknowns": unknowns,
           "initial_guess": {"extrapolate": "4u^{m-1} - 6u^{m-2} + 4u^{m-3} - u^{m-4}",
                             True: "u^{m-1}", False: "0"}[warm]}
    t0 = time.perf_counter()
    best, tried = pkg.batch_tune(inst, M, probe_levels=4, precision="mixed", warm_start=warm, stream=stream,
                                 krylov="auto")
    out["plan"] = best
    out["plans_tried"] = tried
    out["tune_s"] = time.perf_counter() - t0
    us = {}
    # FP64 at 1e-12 drifts by up to 3e-10 over these levels (its recursive
    # residual accumulates per-level errors of ~1e-12 against a huge ahat);
    # at 1e-13 it stays within 2e-11 of a 1e-15 reference, as the mixed path
    # does at 1e-12 (within 2e-13): the arms are compared at equal accuracy.
    tols = {"mixed": 1e-12, "fp64": 1e-13}
    out["krylov_tol"] = tols
    # both Krylov methods on the first levels, in both arithmetics; the faster
    # mixed method then runs the whole march
    def run_one(key, prec, kry, lv, start=warm):
        bs = pkg.BatchSolver(inst, M, precision=prec, stream=stream, warm_start=start,
                             krylov_tol=tols[prec], plan=best, krylov=kry)
        outs = [torch.zeros(d["n"], dtype=torch.float64, device="cuda") for d in inst]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            info = bs.solve(outs, levels=lv)
            e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        out[key] = {"levels": lv, "krylov": kry, "s": t, "instance_levels_per_s": len(inst) * lv / t,
                    "unknown_levels_per_s": unknowns * lv / t,
                    "krylov_its": info["iterations"], "outer": info["outer"],
                    "fp64_levels": info["fp64_levels"], "status": info["status"],
                    "max_final_rel_residual": info["max_rel_residual"]}
        if lv == levels:
            us[key] = [u.cpu().numpy() for u in outs]
        del bs

    # the per-level method choice in both arithmetics, and the paper's FP64
    # BiCGSTAB, on the first levels; the mixed path over the whole march
    run_one("mixed", "mixed", "auto", levels)
    run_one("fp64", "fp64", "auto", levels)
    # the paper's solver from u^{m-1}, as in the headline comparison
    run_one("fp64_paper_bicgstab", "fp64", "bicgstab", levels, start=warm is not False)
    if full:
        run_one("mixed_full_M", "mixed", "auto", M)
    out["mixed_vs_fp64_max_rel_err"] = max(
        float(np.max(np.abs(a - b)) / np.max(np.abs(b))) for a, b in zip(us["mixed"], us["fp64"]))
    out["mixed_speedup"] = out["fp64"]["s"] / out["mixed"]["s"]
    out["mixed_speedup_vs_paper_bicgstab"] = out["fp64_paper_bicgstab"]["s"] / out["mixed"]["s"]
    return out


FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (non-tensor), nominal


def dids_sample(torch, pkg, prob, stream, levels, warm, u_fids_M, krylov):
    """The direct-history scheme DIDS (Eq. (4.1)) on the headline workload
    with the double-single mixed solve: all levels resident, the history sum
    over every earlier level formed by k_rhs_direct.  Times `levels` levels
    from level 1 (CUDA events on the solver's stream; no L2 flush: the
    history read, up to 4.3 GB per level, is far larger than L2) and reports
    the history kernel's algorithmic bytes (8 n m per level m, plus 32 n of
    b, kappa and f) and its FP64 FMA rate (one per history entry)."""
    n = prob.n
    s = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, n, prob.M, prob.r, prob.soe_tol,
                   precision="mixed_ds", krylov_tol=1e-12, profile=True, stream=stream,
                   warm_start=warm, history="direct", krylov=krylov)
    s.set_problem_from(prob)
    with torch.cuda.stream(stream):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(levels):
            s.step(sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    tim = s.timing()
    st = s.level_stats(1, levels)
    hist = sum(m for m in range(1, levels + 1)) * n
    rhs_s = tim["rhs_ms"] / 1e3
    byts = 8.0 * hist + 32.0 * n * levels
    out = {"workload": f"fids-dids n={n} M={prob.M} levels 1..{levels}, mixed_ds {krylov} solve",
           "levels_per_s": levels / t, "s": t,
           "history_kernel": {"ms_per_level": 1e3 * rhs_s / levels,
                              "GB/s": byts / rhs_s / 1e9, "hbm_frac": byts / rhs_s / 1e9 / measured_peaks()[0],
                              "fp64_tflops": 2.0 * hist / rhs_s / 1e12,
                              "fp64_frac_of_nominal": 2.0 * hist / rhs_s / 1e12 / FP64_NOMINAL_TFLOPS},
           "level_kernel_ms_per_level": tim["level_ms"] / levels,
           "iterations_per_level": sum(r["iterations"] for r in st) / levels,
           "max_final_rel_residual": max(r["rel_residual"] for r in st),
           "status": max(r["status"] for r in st)}
    if u_fids_M is not None and levels == prob.M:
        u = torch.empty(n, dtype=torch.float64, device="cuda")
        s.current_solution(u)
        out["dids_vs_fids_max_rel_diff_at_M"] = float(torch.max(torch.abs(u - u_fids_M)) /
                                                      torch.max(torch.abs(u_fids_M)))
    s.close()
    return out


def adjoint_sample(torch, pkg, ti, stream):
    """The adjoint workload: n = 4095, M = 1024, J = 1/2 ||u^M - u_obs||^2
    with u_obs from another kappa.  Times the forward march (FP64) and the
    reverse sweep (transposed FP64 solves, reversed SOE recurrence, fused
    gradient products) twice: over the stored trajectory, and with
    ceil(sqrt(M)) = 32-level checkpoints (u_all = NULL: each segment marched
    again from its checkpoint).  The gradient is checked against central
    differences of J along 3 seeded directions in (kappa, f)."""
    prob, kobs = ti.config_adjoint()
    n, M = prob.n, prob.M
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    s = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, n, M, prob.r, 1e-12, stream=stream,
                   ckpt_stride=-1)
    ones = np.ones(M + 1)
    U = torch.zeros((M + 1, n), dtype=torch.float64, device="cuda")
    uf = torch.zeros(n, dtype=torch.float64, device="cuda")

    def forward(kap, f, keep=True):
        s.set_problem(dev(prob.phi), dev(kap), None, None, F=[dev(f)], G=[ones])
        s.solve(uf, U if keep else None)
        torch.cuda.synchronize()
        return uf

    f0 = prob.F[0]
    u_obs = forward(kobs, f0).clone()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    gk = torch.zeros(n, dtype=torch.float64, device="cuda")
    gf = torch.zeros(n, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        e[0].record(stream)
        forward(prob.kappa0, f0)
        e[1].record(stream)
        info = s.adjoint(U, U[M] - u_obs, gk, gf)
        e[2].record(stream)
        gk2 = torch.zeros_like(gk)
        gf2 = torch.zeros_like(gf)
        info2 = s.adjoint(None, U[M] - u_obs, gk2, gf2)
        e[3].record(stream)
    torch.cuda.synchronize()
    t_fwd = e[0].elapsed_time(e[1]) / 1e3
    t_adj = e[1].elapsed_time(e[2]) / 1e3
    t_ck = e[2].elapsed_time(e[3]) / 1e3
    ck_diff = float(torch.max(torch.abs(gk2 - gk)) / torch.max(torch.abs(gk)))
    gkh, gfh = gk.cpu().numpy(), gf.cpu().numpy()
    J = lambda kap, f: 0.5 * float(torch.sum((forward(kap, f, keep=False) - u_obs) ** 2))
    sk, sf, h = float(np.max(prob.kappa0)), float(np.max(np.abs(f0))), 1e-6
    rng = np.random.default_rng(20)
    worst = 0.0
    for _ in range(3):
        dk = rng.standard_normal(n)
        df = rng.standard_normal(n)
        dk /= np.linalg.norm(dk)
        df /= np.linalg.norm(df)
        fd = (J(prob.kappa0 + h * sk * dk, f0 + h * sf * df) - J(prob.kappa0 - h * sk * dk, f0 - h * sf * df)) / (2 * h)
        ad = sk * (gkh @ dk) + sf * (gfh @ df)
        worst = max(worst, abs(ad - fd) / abs(fd))
    return {"workload": "fids-adjoint n=4095 M=1024 gamma=0.5 alpha=1.4 kappa=lognormal GRF",
            "forward_s": t_fwd, "adjoint_s": t_adj, "adjoint_levels_per_s": M / t_adj,
            "adjoint_checkpointed_s": t_ck, "checkpoint_stride": int(math.ceil(math.sqrt(M))),
            "checkpointed_vs_trajectory_max_rel_diff": ck_diff,
            "recomputed_levels": info2["recomputed_levels"],
            "adjoint_iterations": info["iterations"], "status": info["status"] or info2["status"],
            "fd_directions": 3, "fd_h": h, "grad_vs_central_difference_max_rel": worst}


MID_PAIRS = [(0.3, 0.8), (0.3, 1.2), (0.3, 1.8), (0.7, 0.8), (0.7, 1.2), (0.7, 1.8)]


def mid_sample(torch, pkg, ti, stream, warm):
    """The mid workload: n = 2^14 - 1, M = 2048, six (gamma, alpha) pairs,
    each a whole march timed with CUDA events on the solver's stream (no L2
    flush: the SOE history, ~2 MB x E, exceeds L2), for the default path
    (double-single mixed solve, per-level Krylov choice), FP64 with the
    same choice, both from the same start, and the paper's FP64 BiCGSTAB,
    started from u^{m-1} as in the headline comparison (x0 = 0 when the
    others start from 0)."""
    arms = {"mixed": dict(precision="mixed_ds", krylov="auto", warm_start=warm),
            "fp64": dict(precision="fp64", krylov="auto", warm_start=warm),
            "paper_bicgstab": dict(precision="fp64", krylov="bicgstab", warm_start=warm is not False)}
    rows = []
    tot = {k: [0.0, 0, 0] for k in arms}
    for g, a in MID_PAIRS:
        prob = ti.config_mid(g, a, M=2048)
        row = {"gamma": g, "alpha": a}
        uM = {}
        for name, kw in arms.items():
            s = pkg.Solver(prob.alpha, prob.gamma, prob.l, prob.T, prob.n, prob.M, prob.r, prob.soe_tol,
                           krylov_tol=1e-12, stream=stream, **kw)
            s.set_problem_from(prob)
            u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                s.solve(u, sync=False)
                e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            st = s.level_stats(1, prob.M)
            its = sum(x["iterations"] for x in st)
            row[name] = {"steps_per_s": prob.M / t, "krylov_its_per_s": its / t,
                         "iterations_per_step": its / prob.M,
                         "status": max(x["status"] for x in st)}
            tot[name][0] += t
            tot[name][1] += prob.M
            tot[name][2] += its
            uM[name] = u
            s.close()
        for name in ("mixed", "fp64"):
            row[name + "_vs_paper_bicgstab_max_rel_diff_at_M"] = float(
                torch.max(torch.abs(uM[name] - uM["paper_bicgstab"])) / torch.max(torch.abs(uM["paper_bicgstab"])))
        rows.append(row)
    out = {"workload": "fids-mid n=16383 M=2048, (gamma, alpha) in {0.3,0.7} x {0.8,1.2,1.8}",
           "pairs": rows}
    for name in arms:
        t, steps, its = tot[name]
        out[name + "_steps_per_s"] = steps / t
        out[name + "_krylov_its_per_s"] = its / t
    out["mixed_speedup_vs_fp64"] = out["mixed_steps_per_s"] / out["fp64_steps_per_s"]
    out["mixed_speedup_vs_paper_bicgstab"] = out["mixed_steps_per_s"] / out["paper_bicgstab_steps_per_s"]
    return out


def current_u(torch, s):
    u = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    s.current_solution(u)
    torch.cuda.synchronize()
    return u


def ours(args):
    import torch
    import paper_2002_11978_gb300 as pkg
    import tsfde_inputs as ti
    from paper_2002_11978_gb300 import build

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    prob = ti.config_mixed(n=args.n, M=args.M)
    W = args.warmup
    K = args.steps if args.steps is not None else max(1, prob.M - W)
    stream = torch.cuda.Stream()
    fl = max(1, args.flush_mb) * 1024 * 1024 // 8
    flush = (torch.empty(fl, dtype=torch.float64, device="cuda"),
             torch.zeros(fl, dtype=torch.float64, device="cuda"))
    n = prob.n

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # initial guess of every level solve (the stopping rule is the same)
    start = "zero" if args.cold_start else args.start
    warm = {"extrapolate": "extrapolate", "prev": True, "zero": False}[start]

    # ---- mixed arm: the reported value
    clocks = ClockSampler(torch.cuda.current_device())
    barrier()
    clocks.start()
    ds = args.inner == "ds"
    prec_mx = "mixed_ds" if ds else "mixed"
    kry = args.krylov
    s_mx, ms_mx, tim_mx, st_mx = run_arm(torch, pkg, prob, prec_mx, W, K, flush, stream,
                                         warm=warm, krylov=kry)
    barrier()
    clk = clocks.stop()
    t_mx = max_over_ranks([sum(ms_mx) / 1e3], "cuda")[0]
    u_mx = current_u(torch, s_mx)
    l2_peak = measured_l2_peak(torch, pkg, stream)

    # ---- plain FP64 arm on the same levels: the comparison
    fp64 = None
    if not args.no_fp64:
        s64, ms64, tim64, st64 = run_arm(torch, pkg, prob, "fp64", W, K, flush, stream,
                                         warm=warm, krylov=kry)
        u64 = current_u(torch, s64)
        rel = float(torch.max(torch.abs(u_mx - u64)) / torch.max(torch.abs(u64)))
        t64 = sum(ms64) / 1e3
        fp64 = {"steps_per_s": K / t64, "ms_per_step": 1e3 * t64 / K,
                "max_final_rel_residual_recursive": st64["max_relres"],
                "iterations_per_step": st64["its"] / K, "krylov_its_per_s": st64["its"] / t64,
                "kernel_ms": {"k_rhs": tim64["rhs_ms"] / K, "k_level64": tim64["level_ms"] / K},
                "status": st64["status"],
                "mixed_vs_fp64_max_rel_err_at_last_level": rel,
                "mixed_speedup": (K / t_mx * (1 if world == 1 else 1)) / (K / t64),
                "krylov": kry}
        s64.close()
        if kry != "bicgstab":
            # the paper's solver, FP64 right-preconditioned BiCGSTAB, on the same
            # levels, started from u^{m-1} (x0 = 0 with --cold-start)
            sb, msb, timb, stb = run_arm(torch, pkg, prob, "fp64", W, K, flush, stream,
                                         warm=(start != "zero"), krylov="bicgstab")
            ub = current_u(torch, sb)
            tb = sum(msb) / 1e3
            fp64["paper_bicgstab"] = {
                "steps_per_s": K / tb, "iterations_per_step": stb["its"] / K,
                "level_kernel_ms": timb["level_ms"] / K,
                "mixed_vs_bicgstab_max_rel_err_at_last_level":
                    float(torch.max(torch.abs(u_mx - ub)) / torch.max(torch.abs(ub))),
                "mixed_speedup": tb / t_mx}
            sb.close()

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        se, ms_e2e, _, _ = run_arm(torch, pkg, prob, prec_mx, W, K, flush, stream, e2e=True,
                                    warm=warm, krylov=kry)
        se.close()
        e2e = {"value": world * K / (sum(ms_e2e) / 1e3), "unit": "steps/s",
               "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 8 * n,
               "note": "per level: kappa^m and f^m copied from pinned host, tsfde_step, u^m copied back"}

    # ---- rooflines from the per-kernel CUDA-event totals
    peak, peak_kind = measured_peaks()
    rhs_ms = tim_mx["rhs_ms"] / K
    lvl_ms = tim_mx["level_ms"] / K
    rhs_bytes = (16.0 * n * st_mx["E_active_sum"] + K * 8.0 * n * (3 + 1)) / K
    # inner-vector accesses per inner iteration: 22 for BiCGSTAB, 15 for PCG
    # (4 or 8 bytes per entry), counted per level by the method that solved
    # it; 5 FP64 vector accesses per refinement sweep
    its_p = st_mx["its_pcg"]
    its_b = st_mx["its"] - its_p
    lvl_bytes = ((15 * its_p + 22 * its_b) * (8.0 if ds else 4.0) * n + 40.0 * n * st_mx["outer"]) / K
    kname = ("k_level_mixed_ds" if ds else "k_level_mixed") + {"pcg": "/pcg", "bicgstab": "",
                                                               "auto": "/auto"}[kry]
    rhs_gbs = rhs_bytes / (rhs_ms * 1e-3) / 1e9
    lvl_gbs = lvl_bytes / (lvl_ms * 1e-3) / 1e9
    dom = (kname, lvl_gbs) if lvl_ms >= rhs_ms else ("k_rhs", rhs_gbs)
    if dom[0] == "k_rhs":
        roof = {"kernel": dom[0], "bound": "hbm", "achieved": dom[1], "peak": peak, "unit": "GB/s",
                "frac": dom[1] / peak, "traffic": measured_traffic(dom[0]),
                "peak_source": f"{peak_kind} hbm_gbs"}
    else:
        # the level solve's vectors stay in L2 (DRAM traffic per launch is a
        # small part of its algorithmic bytes), so L2 bounds its bandwidth;
        # its time goes to grid barriers and dependent L2 round trips
        roof = {"kernel": dom[0], "bound": "l2", "achieved": dom[1], "peak": l2_peak, "unit": "GB/s",
                "frac": dom[1] / l2_peak, "traffic": measured_traffic(dom[0]),
                "peak_source": f"measured in this run: tsfde_probe_l2_read over a {L2_PROBE_MB} MB "
                               "L2-resident buffer",
                "hbm_peak": peak, "hbm_frac": dom[1] / peak, "hbm_peak_source": f"{peak_kind} hbm_gbs",
                "note": "latency-bound: about 5 (PCG) or 11 (BiCGSTAB) grid-wide phases per inner "
                        "iteration, each a barrier plus dependent L2 round trips"}

    batched = None
    if args.batched_levels > 0:
        batched = batched_sample(torch, pkg, ti, args.batched_levels, rank, world, stream,
                                 warm=warm, full=not args.no_batched_full)
        if world > 1:
            keys = [k for k in ("mixed", "fp64", "mixed_full_M") if k in batched]
            tm = max_over_ranks([batched[k]["s"] for k in keys], "cuda")
            for k, key in enumerate(keys):
                batched[key]["s_max_over_ranks"] = tm[k]
                batched[key]["instance_levels_per_s"] = 512 * batched[key]["levels"] / tm[k]

    dids = None
    dl = prob.M if args.dids_levels is None else min(args.dids_levels, prob.M)
    if rank == 0 and dl > 0:
        u_f = u_mx if s_mx.m == prob.M else None
        dids = dids_sample(torch, pkg, prob, stream, dl, warm, u_f, kry)

    adjoint = None
    if rank == 0 and not args.no_adjoint:
        adjoint = adjoint_sample(torch, pkg, ti, stream)

    mid = None
    if rank == 0 and not args.no_mid:
        mid = mid_sample(torch, pkg, ti, stream, warm)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(prob, args.cpu_sample_n)
        cpu["all_cores"] = cpu_baseline_sample(prob, args.cpu_sample_n, threads=os.cpu_count() or 1)

    if rank == 0:
        line = {
            "metric": METRIC, "value": world * K / t_mx, "unit": "steps/s", "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": t_mx * 1e3 / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "M": prob.M, "first_timed_level": W + 1,
                       "precision": ("mixed: double-single (FP32-pair) inner " if ds else "mixed: FP32 inner ")
                                    + {"pcg": "PCG on the symmetrised system", "bicgstab": "PBiCGSTAB",
                                       "auto": "per-level choice of PBiCGSTAB or PCG on the symmetrised "
                                               "system (measured level times)"}[kry]
                                    + ", FP64 refinement/residual/SOE",
                       "krylov": kry,
                       "krylov_tol": 1e-12, "inner_tol": 1e-2,
                       "initial_guess": {"extrapolate": "4u^{m-1} - 6u^{m-2} + 4u^{m-3} - u^{m-4} (cubic in the level index)",
                                         "prev": "u^{m-1}", "zero": "0 (Sec. 5)"}[start],
                       "l2": f"flushed before every timed level ({args.flush_mb} MB write, then {args.flush_mb} MB read, outside the events)",
                       "parallelism": f"replicas x{world}"},
            "status": st_mx["status"],
            "iterations_per_step": st_mx["its"] / K, "outer_per_step": st_mx["outer"] / K, "fp64_fallback_levels": st_mx.get("fallback", 0),
            "pcg_levels": st_mx["levels_pcg"], "bicgstab_levels": st_mx["levels"] - st_mx["levels_pcg"],
            "max_final_rel_residual": st_mx["max_relres"], "levels_above_tol": st_mx["above_tol"],
            "krylov_its_per_s": world * st_mx["its"] / t_mx,
            "kernels": {"k_rhs": {"ms": rhs_ms, "bytes": rhs_bytes, "GB/s": rhs_gbs, "frac": rhs_gbs / peak},
                        kname: {"ms": lvl_ms, "bytes": lvl_bytes, "GB/s": lvl_gbs,
                                "frac": lvl_gbs / peak, "l2_frac": lvl_gbs / l2_peak}},
            "fp64": fp64, "e2e": e2e, "gpu_launches": ((3 if kry == "auto" else 2) + (1 if ds else 0)) * K, "roofline": roof,
            "cpu_baseline": cpu, "clocks": clk, "batched": batched, "adjoint": adjoint, "dids": dids, "mid": mid,
        }
        print(json.dumps(line), flush=True)
    s_mx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------ CPU baseline
def cpu_baseline_sample(prob, n_s=2047, budget_s=15.0, threads=1):
    """The oracle (plain C: dense LU with partial pivoting per level, direct
    O(m n) history sums, the FIDS weights summed over the SOE table) on the
    same workload generators at n_s interior points on the full M-level mesh,
    levels 1..k with k sized to the time budget, on `threads` host threads
    (the LU's row updates; the result does not depend on the count).

    Extrapolation to n = prob.n, stated as such: one dense LU of the same
    size is timed on its own; the per-level time splits into that LU
    (scaled by (n/n_s)^3) and the rest (dense level-matrix assembly, O(n^2),
    and the history sums, O(m n) with m << n here; both scaled by
    (n/n_s)^2, an upper bound for the history part).  At n_s = 2047 the LU
    is ~99% of a level, and for the first levels (m < 100) the history and
    weights are < 0.1%, so which window of early levels is sampled does not
    change the figure: both bench arms report this same sample."""
    import oracle
    import tsfde_inputs as ti
    p = ti.config_mixed(n=n_s, M=prob.M)
    tm, tau = oracle.graded_mesh(p.T, p.M, p.r)
    soe = oracle.soe_build(p.gamma, tau[1], p.T, p.soe_tol)
    old_threads = oracle.get_threads()
    oracle.set_threads(threads)
    try:
        K = p.kappa_table(tm)
        F = p.f_table(tm)
        # one dense LU of the level matrix's size and structure
        t = oracle.ifl_symbol(p.alpha, n_s)
        Amat = oracle.dense_A(t) * p.kappa0[:, None] + 1e3 * np.eye(n_s)
        rhs = np.ones(n_s)
        t0 = time.perf_counter()
        oracle.lu_solve(Amat, rhs)
        t_lu = time.perf_counter() - t0
        k = int(max(2, min(64, budget_s / max(t_lu, 1e-6))))
        t0 = time.perf_counter()
        oracle.march("FIDS", p.alpha, p.gamma, p.l, p.T, p.r, p.n, p.M, p.phi, K, F, soe=soe, levels=k)
        el = time.perf_counter() - t0
    finally:
        oracle.set_threads(old_threads)
    per_level = el / k
    rest = max(per_level - t_lu, 0.0)
    q = prob.n / n_s
    ext = t_lu * q ** 3 + rest * q ** 2
    cpu = os.cpu_count() or 1
    return {"value": 1.0 / ext, "unit": "steps/s", "cores": threads, "kind": "oracle",
            "sample": (f"oracle FIDS (dense LU per level, direct history sums, SOE E={len(soe[0])}) on the "
                       f"same generators at n={n_s}, levels 1..{k} of M={p.M}, {threads} thread(s) of {cpu}: "
                       f"{per_level:.3f} s per level, of which one dense LU {t_lu:.3f} s; extrapolated to "
                       f"n={prob.n} as LU x (n/n_s)^3 + rest x (n/n_s)^2 = {ext:.3g} s per level"),
            "extrapolated": True, "sample_n": n_s, "sample_levels": k, "sample_s_per_level": per_level,
            "sample_lu_s": t_lu, "host_cpus": cpu}


def reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import tsfde_inputs as ti
    prob = ti.config_mixed(n=args.n, M=args.M)
    W = args.warmup
    K = args.steps if args.steps is not None else max(1, prob.M - W)
    K = min(K, prob.M - W)
    cpu = cpu_baseline_sample(prob, args.cpu_sample_n)
    cpu["all_cores"] = cpu_baseline_sample(prob, args.cpu_sample_n, threads=os.cpu_count() or 1)
    line = {"metric": METRIC, "value": cpu["value"], "unit": "steps/s", "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": 1e3 / cpu["value"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "n": prob.n, "M": prob.M, "first_timed_level": W + 1,
                       "parallelism": "one host thread (all-core run in cpu_baseline.all_cores)"},
            "cpu_baseline": cpu,
            "e2e": {"value": cpu["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        reference(a)
    else:
        ours(a)
