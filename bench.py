#!/usr/bin/env python3
"""Benchmark of the GB300 Stokes solver: solves/s at relres 1e-8.

One step = one complete solve of the workload (gather, preconditioned MINRES
with the inner IC(0)-CG preconditioner, true residual, zero-mean pressure
filter, scatter) on inputs already resident in HBM.  The problem set-up
(patterns, assembly, IC(0) factorisation) is done once before the timed
region, like the paper's separate R+F column.  The default workload is the
largest single-GPU configuration: 2D, 1024 x 1024 elements, velocity degree 3
(k' = 2), FP64, one right-hand side, Diag(Q_nu) pressure block.

Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbs|reference]
                  [--workload 2d1024|2d256|2d256p4|2d16|3d32|3d48|cavity256]
Under torchrun (N > 1) each rank solves its own forcings on its own GPU
(replicas: the method has no data-parallel exchange); the value is the total
number of solves over the slowest rank's time.  --impl reference times the
FP64 CPU oracle (the only other implementation there is) on bounded samples.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Stokes solves/s at relres 1e-8, plain FP64 vs mixed/batched; SpMV HBM GB/s"

WORKLOADS = {
    "2d256": dict(dim=2, N=256, p=3, desc="2D unit square, 256x256 elements, velocity degree 3 / pressure degree 2 "
                                          "(k'=2), nu=1, Nitsche no-slip, 16-mode seeded Fourier forcing"),
    "2d256p4": dict(dim=2, N=256, p=4, desc="2D unit square, 256x256 elements, k'=3, nu=1, 16-mode Fourier forcing"),
    "2d16": dict(dim=2, N=16, p=3, desc="2D unit square, 16x16 elements, k'=2, nu=1, 16-mode Fourier forcing"),
    "3d32": dict(dim=3, N=32, p=3, desc="3D unit cube, 32^3 elements, k'=2, nu=1, 16-mode Fourier forcing"),
    "2d1024": dict(dim=2, N=1024, p=3, desc="2D unit square, 1024x1024 elements, k'=2, nu=1, Fourier forcing"),
    # the same kernels on a quarter of the unknowns (profiling captures that must stay small)
    "2d512": dict(dim=2, N=512, p=3, desc="2D unit square, 512x512 elements, k'=2, nu=1, Fourier forcing"),
    "3d48": dict(dim=3, N=48, p=3, desc="3D unit cube, 48^3 elements, k'=2, nu=1, Fourier forcing"),
    # the paper's own benchmark problem (Sec. 6.4); run it as in Table ic_pgc_tols_k2 with
    # --pressure pcg --tol 1e-12 --inner-tol 1e-3
    "cavity256": dict(dim=2, N=256, p=3, load="cavity",
                      desc="2D lid-driven cavity, 256x256 elements, k'=2, nu=1, unit lid velocity (Nitsche load)"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gbs", "reference"], default="gbs")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="2d1024")
    ap.add_argument("--ordering", choices=["natural", "rcm", "multicolour"], default="multicolour")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--spmv", choices=["auto", "csr", "sell", "sell2w", "sell4w"], default="auto",
                    help="single-RHS SpMV layout of the benchmark precision (auto: timed at the first solve)")
    ap.add_argument("--trsv", choices=["auto", "csr", "sell", "staged4", "staged12", "staged32", "packed12",
                                       "packed32", "split12", "split32", "sellw", "tma", "sellwl", "sellwl8", "sellwlr", "sellwl32", "sellwl2",
                                       "sellwl24", "sellwl48", "sellwlh"],
                    default="auto",
                    help="single-RHS IC(0) sweep layout of the benchmark precision")
    ap.add_argument("--stop", choices=["residual", "estimate"], default="residual",
                    help="MINRES stop: ||b - Kx|| / ||b|| <= tol (the paper's relative residual) or |eta| / gamma_1")
    ap.add_argument("--pressure", choices=["diag", "pcg"], default="diag",
                    help="pressure block: Diag(Q_nu) or IC(0)-PCG on Q_nu (Sec. 6.4)")
    ap.add_argument("--k", type=int, default=1, help="right-hand sides per solve")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--inner-tol", type=float, default=1e-2)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--all-variants", action="store_true",
                    help="also the 3D 48^3 x 32 batches with the Diag(Q_nu) pressure block")
    ap.add_argument("--e2e-steps", type=int, default=2,
                    help="solves timed end to end through gb_solve_host (each one a full solve)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--max-outer", type=int, default=5000,
                    help="MINRES iteration cap (lowered only for short profiling runs)")
    a = ap.parse_args()
    if a.warmup < 3:
        a.warmup = 3
    return a


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, dist=None, device="cuda"):
    """The largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(world, steps, k, ms_slowest):
    """Whole-job solves/s: every rank solves `steps` batches of k right-hand
    sides; the job takes as long as the slowest rank."""
    return world * steps * k / (ms_slowest / 1000.0)


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms in the background."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _definition(path, name):
    """Source text of the function `name` in `path`: its definition (an
    occurrence of `name(` outside a line comment whose parameter list is
    followed by a body), from the line that declares it (and a template line
    right above) to the brace that closes its body; "" if there is none."""
    with open(path) as fh:
        src = fh.read()
    pos = 0
    while True:
        i = src.find(name + "(", pos)
        if i < 0:
            return ""
        pos = i + 1
        line_start = src.rfind("\n", 0, i) + 1
        if "//" in src[line_start:i] or (i > 0 and (src[i - 1].isalnum() or src[i - 1] == "_")):
            continue  # in a comment, or the tail of a longer name
        k, depth = i + len(name), 0
        while k < len(src):
            depth += {"(": 1, ")": -1}.get(src[k], 0)
            k += 1
            if depth == 0:
                break
        rest = src[k:].lstrip()
        while rest.startswith("const") or rest.startswith("noexcept"):
            rest = rest.split(None, 1)[1] if " " in rest else ""
        if not rest.startswith("{"):
            continue  # a declaration or a call
        prev = src.rfind("\n", 0, max(line_start - 1, 0)) + 1
        start = prev if line_start > 0 and src[prev:line_start].lstrip().startswith("template") else line_start
        j = src.find("{", k)
        depth = 0
        for m in range(j, len(src)):
            depth += {"{": 1, "}": -1}.get(src[m], 0)
            if depth == 0:
                return src[start:m + 1]
        return src[start:]


# (kernel, sweep layout family) -> (file, function) pairs whose text decides
# the DRAM traffic of a launch
TRAFFIC_SOURCES = {
    ("ic0_apply", "packed"): [("solver_kernels.cuh", "k_trsv_level_packed"), ("setup.cpp", "build_packed")],
    ("ic0_apply", "split"): [("solver_kernels.cuh", "k_trsv_level_split"), ("setup.cpp", "build_packed")],
    ("ic0_apply", "sellwl"): [("solver_kernels.cuh", "k_trsv_level_sellw"), ("layouts.cpp", "sell_layout")],
    ("ic0_apply", "sellwlr"): [("solver_kernels.cuh", "k_trsv_level_sellw"), ("layouts.cpp", "sell_layout")],
    ("ic0_apply", "sellw"): [("solver_kernels.cuh", "k_trsv_level_sellw"), ("layouts.cpp", "sell_layout")],
    ("ic0_apply", "sellwlh"): [("solver_kernels.cuh", "k_trsv_level_sellw"), ("layouts.cpp", "sell_layout")],
}


def _layout_family(trsv):
    """'packed32' -> 'packed', 'split12' -> 'split' (None stays None)."""
    return trsv.rstrip("0123456789") if trsv else trsv


def source_hash(kernel="ic0_apply", trsv="packed32"):
    """Hash of the source of the kernel (and of the layout it reads) whose
    ncu traffic is recorded for this sweep layout; a change there
    invalidates the record.  None if no sources are registered."""
    srcs = TRAFFIC_SOURCES.get((kernel, _layout_family(trsv)))
    if not srcs:
        return None
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1309_5048_gb300", "csrc")
    for fname, func in srcs:
        h.update(_definition(os.path.join(csrc, fname), func).encode())
    return h.hexdigest()[:16]


def traffic_for(kernel, workload, trsv=None, precision=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources with the same sweep layout and precision;
    else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("precision") != precision:
        return None
    # a record may name several layouts that read the same data (e.g. the same
    # kernel on two grid sizes)
    names = e.get("trsv")
    if trsv not in (names if isinstance(names, list) else [names]):
        return None
    h = source_hash(kernel, trsv)
    if h is None or e.get("src_hash") != h:
        return None
    return e.get("dram_bytes_per_launch")


def algorithmic_bytes(s, kernel, precision, k):
    """Bytes the method must move per launch (each stored nonzero read once
    as value + 32-bit index, each vector operand read or written once)."""
    vb = 4 if precision == "mixed" else 8
    mb = vb + 4
    nnzL = s.nnzL  # includes the diagonal (stored as its inverse)
    if kernel == "cg_spmv":  # q = A p, p^T q: matrix + p gather + q write + row pointers
        return mb * s.nnzA + k * (2 * vb) * s.n_u + 4 * s.n_u
    if kernel == "ic0_apply":  # L y = r then L^T z = y
        one = mb * nnzL + k * (2 * vb) * s.n_u + 4 * s.n_u
        return 2 * one
    if kernel == "stokes_apply":  # A, B^T, B in FP64 + z gather + q write
        return 12 * (s.nnzA + 2 * s.nnzB) + k * 16 * s.n + 4 * (s.n_u + s.n)
    raise ValueError(kernel)


def cg_vector_bytes(s, precision):
    """Vector bytes of one inner CG iteration beyond its SpMV and IC(0)
    application: nine n_u-vector reads or writes (x and r updates, r^T z,
    p update)."""
    return 9 * (4 if precision == "mixed" else 8) * s.n_u


def minres_vector_bytes(s):
    """FP64 vector bytes of one MINRES step beyond its Stokes product and
    preconditioner application: fourteen (n_u + n_p)-vector reads or writes
    (Lanczos, rotation, w and x updates) and three n_p ones (Diag(Q) scaling,
    zero-mean pressure)."""
    return 14 * 8 * (s.n_u + s.n_p) + 3 * 8 * s.n_p


def solve_bytes(s, info, precision):
    """Algorithmic bytes of one single-RHS solve with the Diag(Q) pressure
    block, from its measured counts: outer + 1 Stokes products, one IC(0)
    application per preconditioner application and per inner iteration, one
    SpMV per inner iteration, and the vector work of both loops."""
    return ((info["outer_its"] + 1) * algorithmic_bytes(s, "stokes_apply", precision, 1)
            + (info["precond_apps"] + info["inner_its_total"]) * algorithmic_bytes(s, "ic0_apply", precision, 1)
            + info["inner_its_total"] * (algorithmic_bytes(s, "cg_spmv", precision, 1) + cg_vector_bytes(s, precision))
            + info["outer_its"] * minres_vector_bytes(s))


def launches_per_solve(s, info, pressure="diag"):
    """Kernel launches of one solve as the graph driver issues them (the
    pressure CG adds, per application, dim line-solve passes and a rho
    kernel, and per iteration an SpMV, an axpy, dim passes, rho, p-update)."""
    L = s.nlevels
    n = (4 + 3 * info["outer_its"] + info["precond_apps"] * (2 * L + 2)
         + info["inner_its_total"] * (2 * L + 4))
    if pressure == "pcg":
        n += info["precond_apps"] * (s.dim + 1) + info["q_inner_its_total"] * (s.dim + 4)
    return n


def oracle_load(P, W, seed=0):
    """The workload's load vector from the oracle (forcing seed `seed`)."""
    from paper_1309_5048_gb300.inputs import fourier_modes
    if W.get("load") == "cavity":
        return P.load_cavity()
    kappa, amp = fourier_modes(W["dim"], seed=seed)
    return P.load_fourier(kappa, amp)


def cpu_model():
    """The host CPU's model name (lscpu), for the record of a CPU timing."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_problem(W, ordering, pressure="diag"):
    """The oracle's problem for a workload: assembled, ordered, factored."""
    import oracle
    P = oracle.Problem(W["dim"], W["N"], W["p"], ordering=ordering)
    P.factor()
    if pressure == "pcg":
        P.factor_q()
    return P


def oracle_rates(P, b_u, inner_tol, target_s, pressure="diag", stop="residual", repeats=1):
    """Oracle cost per unit of solve work, timed on the workload itself:
    * t_inner: seconds per inner CG iteration (one SpMV with A_h, the forward
      and backward IC(0) sweeps and the CG vector updates), from an inner PCG
      on the workload's first preconditioner input b_u (the velocity part of
      the right-hand side) run for about target_s seconds;
    * t_step, t_fixed: seconds per MINRES step and once per solve when every
      preconditioner application does exactly one inner iteration (the
      oracle's replay mode forces the count): the Stokes products, the
      residual test, the Lanczos and update vector work, the IC(0)
      application that starts each inner CG and its single iteration; from
      two such runs, of one step and of about target_s / 2 seconds.
    Each timing is the fastest of `repeats` runs (a busy host only adds
    time)."""
    import numpy as np
    b = np.concatenate([b_u, np.zeros(P.n_p)])
    t = time.perf_counter()
    P.pcg(b_u, inner_tol=1e-300, max_inner=2)
    pilot = (time.perf_counter() - t) / 2
    m = int(max(3, min(20000, target_s / max(pilot, 1e-9))))
    dts = []
    for _ in range(repeats):
        t = time.perf_counter()
        _, its = P.pcg(b_u, inner_tol=1e-300, max_inner=m)
        dts.append(time.perf_counter() - t)
    dt = min(dts)
    def forced_run(steps):
        t = time.perf_counter()
        P.minres(b, tol=1e-300, inner_tol=inner_tol, max_outer=steps, forced=[1] * (steps + 1),
                 forced_q=[1] * (steps + 1) if pressure == "pcg" else None, pressure=pressure, stop=stop)
        return time.perf_counter() - t

    t1 = min(forced_run(1) for _ in range(repeats))
    n2 = int(max(3, min(2000, target_s / 2.0 / max(t1, 1e-9))))  # about target_s / 2 seconds
    t2 = min(forced_run(n2) for _ in range(repeats))
    t_step = max((t2 - t1) / (n2 - 1), 0.0)
    return {"t_inner": dt / max(its, 1), "t_step": t_step, "t_fixed": max(t1 - t_step, 0.0),
            "its": int(its), "steps": n2, "seconds": repeats * (dt + t1 + t2)}


def oracle_solve_seconds(rates, counts):
    """Oracle time of a whole solve from its work counts: a one-inner-
    iteration MINRES step per step (t_step, plus t_fixed once), and the
    remaining inner CG iterations at t_inner each."""
    extra = counts["inner_its_total"] - counts["precond_apps"]
    return rates["t_fixed"] + rates["t_step"] * counts["outer_its"] + rates["t_inner"] * max(extra, 0)


COUNTS_PATH = os.path.join(ROOT, "profiles", "solve_counts.json")


def recorded_counts(workload, key):
    """Work counts (outer_its, precond_apps, inner_its_total) of a full FP64
    solve recorded for a workload and solver setting, or None."""
    try:
        with open(COUNTS_PATH) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    return d.get(workload, {}).get(key)


def counts_key(precision, pressure, tol, inner_tol, stop, k=1):
    return "%s_%s_tol%g_inner%g_%s_k%d" % (precision, pressure, tol, inner_tol, stop, k)


def cpu_baseline(P, W, b_u, counts, inner_tol, target_s=15.0, pressure="diag", stop="residual"):
    """The oracle as it stands, single-threaded, on a bounded sample of the
    same workload (oracle_rates), scaled by the work counts of the full solve
    measured on the GPU in this run (oracle_solve_seconds)."""
    r = oracle_rates(P, b_u, inner_tol, target_s, pressure, stop)
    est = oracle_solve_seconds(r, counts)
    return {"value": 1.0 / est, "unit": "solves/s", "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": ("oracle on this workload (forcing seed 0), %.1f s of samples: %d inner CG iterations "
                       "(%.3g s each) and MINRES runs of 1 and %d steps with one inner iteration per "
                       "preconditioner application (%.3g s per step), scaled to a full solve by its counts "
                       "(%d MINRES steps, %d preconditioner applications, %d inner CG iterations, from the GPU "
                       "solve of the same system): %.0f s per solve; oracle assembly/ordering/IC(0) excluded"
                       % (r["seconds"], r["its"], r["t_inner"], r["steps"], r["t_step"], counts["outer_its"],
                          counts["precond_apps"], counts["inner_its_total"], est))}


def run_reference(args):
    """--impl reference: the FP64 CPU oracle, each step a bounded sample (an
    inner PCG of the workload), scaled to solves/s by the work counts of the
    full solve (oracle_solve_seconds)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    W = WORKLOADS[args.workload]
    P = oracle_problem(W, args.ordering, args.pressure)
    b_u = oracle_load(P, W)
    b = np.concatenate([b_u, np.zeros(P.n_p)])
    key = counts_key("fp64", args.pressure, args.tol, args.inner_tol, args.stop)
    counts = recorded_counts(args.workload, key)
    source = "recorded in profiles/solve_counts.json (GPU FP64 solve of the same system)"
    full_s = None
    if counts is None:
        # small workloads: the oracle's own full solve gives the counts, and
        # its time is printed beside the estimate
        t = time.perf_counter()
        _, full = P.minres(b, tol=args.tol, inner_tol=args.inner_tol, pressure=args.pressure, stop=args.stop)
        full_s = time.perf_counter() - t
        counts = {"outer_its": full["outer"], "precond_apps": int(len(full["counts"])),
                  "inner_its_total": int(np.sum(full["counts"]))}
        source = "from the oracle's own full solve, which took %.1f s" % full_s
    per_step = max(0.5, min(6.0, 120.0 / max(args.steps + args.warmup, 1)))
    for _ in range(args.warmup):
        oracle_rates(P, b_u, args.inner_tol, per_step, args.pressure, args.stop)
    t = time.perf_counter()
    samples = [oracle_rates(P, b_u, args.inner_tol, per_step, args.pressure, args.stop) for _ in range(args.steps)]
    dt = time.perf_counter() - t
    rates = {k_: statistics.median(r[k_] for r in samples) for k_ in ("t_inner", "t_step", "t_fixed")}
    est = oracle_solve_seconds(rates, counts)
    value = 1.0 / est
    sample = ("each step: an inner PCG of ~%.1f s on this workload's first preconditioner input and two MINRES "
              "runs with one inner iteration per preconditioner application; medians %.3g s per "
              "inner CG iteration, %.3g s per MINRES step, scaled to a full solve by its counts (%d MINRES "
              "steps, %d preconditioner applications, %d inner CG iterations; %s): %.0f s per solve"
              % (per_step, rates["t_inner"], rates["t_step"], counts["outer_its"], counts["precond_apps"],
                 counts["inner_its_total"], source, est))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * dt / max(args.steps, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W["desc"], "ordering": args.ordering, "k": 1, "precision": "fp64",
                       "tol": args.tol, "inner_tol": args.inner_tol,
                       "pressure_block": "Diag(Q)" if args.pressure == "diag" else "IC(0)-PCG(Q)",
                       "stop": args.stop},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "cpu_model": cpu_model(), "sample": sample, "estimate_s": est,
                             "full_solve_s": full_s},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "counts": counts}
    print(json.dumps(line), flush=True)
    return 0


def oracle_rows(W, s, nrows_u=400, nrows_p=200, seed=5):
    """The oracle's own rows of A_h and B (assembled for sampled rows only)
    for a residual check of GPU solutions at sizes the oracle cannot solve:
    sampled velocity rows ru, and pressure rows rp = every pressure row
    coupled to ru (so that (B^T x_p)_i is complete for i in ru) plus random
    ones.  Returns a function x (natural numbering, n) -> (r_u rows, r_p rows)
    of b - K x, and the row counts."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(seed)
    ru = np.sort(rng.choice(s.n_u, nrows_u, replace=False))
    ptrB, colB, _ = s.csr("B")  # the pattern only, to find the coupled pressure rows
    rowsB = np.repeat(np.arange(s.n_p), np.diff(ptrB))
    mark = np.zeros(s.n_u, bool)
    mark[ru] = True
    coupled = np.unique(rowsB[mark[colB]])
    extra = rng.choice(s.n_p, nrows_p, replace=False)
    rp = np.union1d(coupled, extra)
    del ptrB, colB, rowsB
    mu = np.zeros(s.n_u, np.int8)
    mp = np.zeros(s.n_p, np.int8)
    mu[ru] = 1
    mp[rp] = 1
    ref = oracle.Problem(W["dim"], W["N"], W["p"], nu=1.0, rows_u=mu, rows_p=mp)
    A = ref.scipy("A").tocsr()[ru]
    B = ref.scipy("B").tocsr()[rp]
    Bu = B[:, ru].tocsc()  # B^T restricted to the sampled velocity rows: (B^T x_p)_i = sum_k B_ki x_p,k

    def residual(b, x):
        xu, xp = x[: s.n_u], x[s.n_u:]
        r_u = b[ru] - A @ xu - Bu.T @ xp[rp]
        r_p = b[s.n_u + rp] - B @ xu
        return r_u, r_p

    return residual, len(ru), len(rp), int(s.n_u), int(s.n_p)


def sampled_relres(check, b, x):
    """The relative residual ||b - K x|| / ||b|| estimated from the oracle's
    sampled rows (each block's mean square scaled to its size)."""
    import numpy as np
    residual, mu, mp, n_u, n_p = check
    r_u, r_p = residual(b, x)
    est = np.sqrt(n_u / mu * float(r_u @ r_u) + n_p / mp * float(r_p @ r_p))
    return est / float(np.linalg.norm(b))


# Variants reported beside the benchmark line (rank 0, one timed solve each,
# after a two-step solve that runs the layout tuning and builds the graph):
# (name, workload or None for the benchmark's, precision, k, pressure block,
# inner tolerance or None for the benchmark's, MINRES cap or None).
VARIANTS = [
    ("mixed_k1", None, "mixed", 1, "diag", None, None),
    ("mixed_k1_inner1e-1", None, "mixed", 1, "diag", 1e-1, 150),
    ("mixed_k1_inner1e-3", None, "mixed", 1, "diag", 1e-3, None),
    ("mixed_k1_inner1e-4", None, "mixed", 1, "diag", 1e-4, None),
    ("fp64_k1_pcgq", None, "fp64", 1, "pcg", None, None),
    ("mixed_k1_pcgq", None, "mixed", 1, "pcg", None, None),
    ("3d48_fp64_k32_pcgq", "3d48", "fp64", 32, "pcg", None, None),
    ("3d48_mixed_k32_pcgq", "3d48", "mixed", 32, "pcg", None, None),
]
# with --all-variants (each about a minute: with Diag(Q_nu) the batch runs
# until its slowest forcing has converged, 230+ MINRES steps in 3D)
EXTRA_VARIANTS = [
    ("3d48_fp64_k32", "3d48", "fp64", 32, "diag", None, None),
    ("3d48_mixed_k32", "3d48", "mixed", 32, "diag", None, None),
]


def rel_diff(a, b):
    import numpy as np
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = dist_env()
    W = WORKLOADS[args.workload]
    # the oracle's problem for the CPU baseline is assembled in a background
    # thread (the oracle's C++ runs outside the GIL) while the GPU works
    cpu_job = {}
    cpu_thread = None
    if rank == 0 and world == 1 and not args.no_cpu:
        def build_oracle():
            try:
                P = oracle_problem(W, args.ordering, args.pressure)
                cpu_job["P"] = P
                cpu_job["b_u"] = oracle_load(P, W)
            except Exception as e:  # reported in the line
                cpu_job["error"] = repr(e)
        cpu_thread = threading.Thread(target=build_oracle, daemon=True)
        cpu_thread.start()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    import paper_1309_5048_gb300 as gb
    from paper_1309_5048_gb300.inputs import fourier_modes

    def make_problem(W_):
        t0 = time.perf_counter()
        s_ = gb.Stokes(W_["dim"], W_["N"], W_["p"], ordering=args.ordering)
        t_setup_ = time.perf_counter() - t0
        t0 = time.perf_counter()
        s_.assemble(1.0)
        s_.factor_ic0()
        torch.cuda.synchronize()
        return s_, t_setup_, time.perf_counter() - t0

    s, t_setup, t_rf = make_problem(W)
    if args.spmv != "auto" or args.trsv != "auto":
        s.set_kernel_variants(args.precision, args.spmv, args.trsv)
    k = args.k

    def make_rhs(s_, W_, k_, seed0):
        rhs_ = torch.zeros(k_, s_.n, dtype=torch.float64, device="cuda")
        for t in range(k_):
            if W_.get("load") == "cavity":  # column t: lid speed 1 + t + seed0 / 1000
                rhs_[t, : s_.n_u] = s_.load_cavity() * (1.0 + t + seed0 / 1000.0)
            else:
                kap, amp = fourier_modes(W_["dim"], seed=seed0 + t)
                rhs_[t, : s_.n_u] = s_.load_fourier(kap, amp)
        return rhs_

    rhs = make_rhs(s, W, k, rank * 1000)
    out = torch.empty_like(rhs)
    opts = dict(tol=args.tol, inner_tol=args.inner_tol, precision=args.precision, use_graph=not args.no_graph,
                max_outer=args.max_outer, pressure=args.pressure, stop=args.stop)

    clocks = ClockSampler(local)
    for _ in range(args.warmup):
        _, info = s.solve(rhs, out=out, **opts)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        _, info = s.solve(rhs, out=out, **opts)
    e1.record()
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    infos = info if isinstance(info, list) else [info]
    value = throughput(world, args.steps, k, ms)
    x_main = out.cpu().numpy().reshape(k, -1)
    b_main = rhs.cpu().numpy().reshape(k, -1)

    # end to end through the public host-buffer call (pinned memory): every
    # step copies the right-hand side in and the solution out
    rhs_h = rhs.cpu().pin_memory()
    out_h = torch.empty_like(rhs_h).pin_memory()
    e2e_steps = max(1, args.e2e_steps)
    barrier()
    t = time.perf_counter()
    for _ in range(e2e_steps):
        s.solve_host(rhs_h, out_h, **opts)
    e2e_s = max_over_ranks(time.perf_counter() - t, dist)
    bytes_io = 8 * k * s.n

    # per-kernel timing (events on the library's stream) and the roofline
    _, info1 = s.solve(rhs, out=out, **opts)
    inf0 = info1[0] if isinstance(info1, list) else info1
    kern = {}
    for name, reps in (("cg_spmv", 50), ("ic0_apply", 20), ("stokes_apply", 50)):
        ms_k = s.time_kernel(name, reps)
        ab = algorithmic_bytes(s, name, args.precision, k)
        kern[name] = {"ms_per_launch": ms_k, "algorithmic_bytes": ab, "gbs": ab / (ms_k * 1e-3) / 1e9}
    count = {"cg_spmv": inf0["inner_its_total"], "ic0_apply": inf0["precond_apps"] + inf0["inner_its_total"],
             "stokes_apply": inf0["outer_its"] + 1}
    for name in kern:
        kern[name]["launches_per_solve"] = count[name]
        kern[name]["est_ms_per_solve"] = count[name] * kern[name]["ms_per_launch"]
    dom = max(kern, key=lambda n: kern[n]["est_ms_per_solve"])
    peak, peak_kind = measured_peak()
    layouts = dict(zip(("spmv", "trsv"), s.kernel_variants(args.precision)))
    roof = {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["gbs"], "peak": peak, "unit": "GB/s",
            "frac": kern[dom]["gbs"] / peak, "peak_source": peak_kind,
            "traffic": traffic_for(dom, args.workload, layouts["trsv"], args.precision),
            "unit_of_launch": ("one preconditioner application: forward + backward IC(0) sweep over %d levels "
                               "each" % s.nlevels) if dom == "ic0_apply" else "one kernel launch"}
    # the whole solve against the same peak: algorithmic bytes from the
    # measured counts over the measured time per solve (k = 1, Diag(Q) only)
    whole = None
    if k == 1 and args.pressure == "diag":
        sb = solve_bytes(s, infos[0], args.precision)
        gbs = sb / (ms / args.steps * 1e-3) / 1e9
        whole = {"bytes_per_solve": sb, "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                 "peak_source": peak_kind}

    # the error of the benchmark solution against the oracle: at sizes the
    # oracle solves whole, the relative solution difference from an oracle
    # solve at tol 1e-13; otherwise the relative residual ||b - K x|| / ||b||
    # estimated on the oracle's own sampled rows of A_h and B
    err_main = None
    check = None
    if rank == 0 and k == 1 and W.get("load") != "cavity":
        try:
            check = oracle_rows(W, s)
            err_main = {"kind": "oracle sampled rows: relres estimate", "rows_u": check[1], "rows_p": check[2],
                        "relres": sampled_relres(check, b_main[0], x_main[0])}
        except Exception as e:  # the line still prints
            err_main = {"kind": "unavailable", "why": repr(e)}

    variants = {}
    if not args.no_variants and rank == 0:
        others = {}
        for name, wl, prec, kk, pres, itol, cap in VARIANTS + (EXTRA_VARIANTS if args.all_variants else []):
            Wv = WORKLOADS[wl] if wl else W
            if wl and wl != args.workload:
                if wl not in others:
                    others.clear()  # one extra problem resident at a time
                    torch.cuda.empty_cache()
                    others[wl] = make_problem(Wv)[0]
                sv = others[wl]
            else:
                sv = s
            r = make_rhs(sv, Wv, kk, 0)
            o = torch.empty_like(r)
            ov = dict(tol=args.tol, inner_tol=itol if itol else args.inner_tol, precision=prec,
                      use_graph=not args.no_graph, pressure=pres, stop=args.stop,
                      max_outer=cap if cap else args.max_outer)
            sv.solve(r, out=o, **dict(ov, max_outer=2))  # layout tuning and graph build
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record()
            _, inf_v = sv.solve(r, out=o, **ov)
            ev1.record()
            torch.cuda.synchronize()
            ms_v = ev0.elapsed_time(ev1)
            iv = inf_v if isinstance(inf_v, list) else [inf_v]
            xv = o.cpu().numpy().reshape(kk, -1)
            entry = {"solves_per_s": kk / (ms_v / 1000.0), "workload": Wv["desc"], "k": kk, "precision": prec,
                     "pressure_block": "Diag(Q)" if pres == "diag" else "IC(0)-PCG(Q)",
                     "inner_tol": ov["inner_tol"], "outer_its_mean": statistics.mean(i["outer_its"] for i in iv),
                     "inner_its_mean": statistics.mean(i["inner_its_total"] for i in iv),
                     "relres_true_max": max(i["relres_true"] for i in iv),
                     "converged": all(i["status"] == 0 for i in iv)}
            if cap:
                entry["max_outer"] = cap
            err = {}
            if sv is s and kk == 1 and k >= 1:
                err["rel_diff_vs_fp64_line"] = rel_diff(xv[0], x_main[0])
                if check is not None:
                    err["oracle_rows_relres"] = sampled_relres(check, b_main[0], xv[0])
            elif kk > 1 and prec != "fp64":
                ref_name = name.replace("mixed", "fp64")
                if ref_name in variants and "_x" in variants[ref_name]:
                    xr = variants[ref_name]["_x"]
                    err["max_rel_diff_vs_fp64_batch"] = max(rel_diff(xv[t], xr[t]) for t in range(kk))
            entry["err_vs_oracle"] = err or None
            if kk > 1 and prec == "fp64":
                entry["_x"] = xv
            variants[name] = entry
        for v in variants.values():
            v.pop("_x", None)
        others.clear()

    cpu = None
    if cpu_thread is not None:
        cpu_thread.join()
        if "error" in cpu_job:
            cpu = {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle", "error": cpu_job["error"]}
        else:
            cnt = {kk_: int(infos[0][kk_]) for kk_ in ("outer_its", "precond_apps", "inner_its_total")}
            cpu = cpu_baseline(cpu_job["P"], W, cpu_job["b_u"], cnt, args.inner_tol, pressure=args.pressure,
                               stop=args.stop)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
            "data": "synthetic",
            "config": {"workload": W["desc"], "ordering": args.ordering, "k": k, "precision": args.precision,
                       "pressure_block": "Diag(Q)" if args.pressure == "diag" else "IC(0)-PCG(Q)",
                       "stop": ("||b - K x||_2 / ||b||_2 <= tol" if args.stop == "residual"
                                else "|eta| / gamma_1 <= tol"),
                       "tol": args.tol, "inner_tol": args.inner_tol, "graph": not args.no_graph,
                       "l2": "no flush: per-iteration working set (A, L, L^T, vectors) exceeds the 129 MB L2",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof,
            "solve_roofline": whole,
            "cpu_baseline": cpu,
            "e2e": {"value": throughput(world, e2e_steps, k, 1000.0 * e2e_s), "unit": "solves/s",
                    "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io, "steps": e2e_steps},
            "gpu_launches": int(args.steps * sum(launches_per_solve(s, i, args.pressure) for i in infos)),
            "clocks": clock_info,
            "outer_its": infos[0]["outer_its"], "inner_its_total": infos[0]["inner_its_total"],
            "precond_apps": infos[0]["precond_apps"],
            "inner_its_mean": infos[0]["inner_its_total"] / max(infos[0]["precond_apps"], 1),
            "relres_est": infos[0]["relres_est"], "relres_true": infos[0]["relres_true"],
            "err_vs_oracle": err_main,
            "setup_s": t_setup, "assemble_factor_s": t_rf, "levels": s.nlevels, "layouts": layouts,
            "kernels": kern, "variants": variants,
            "variants_note": "one timed solve each (after a two-step tuning solve); 3D 48^3 uses forcing seeds 0-31",
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
