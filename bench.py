#!/usr/bin/env python3
"""Benchmark of the GB300 Stokes solver: solves/s at relres 1e-8.

One step = one complete solve of the workload (gather, preconditioned MINRES
with the inner IC(0)-CG preconditioner, true residual, zero-mean pressure
filter, scatter) on inputs already resident in HBM.  The problem set-up
(patterns, assembly, IC(0) factorisation) is done once before the timed
region, like the paper's separate R+F column.

Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbs|reference]
                  [--workload 2d256|2d256p4|2d16|3d32|2d1024|3d48]
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
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="2d256")
    ap.add_argument("--ordering", choices=["natural", "rcm", "multicolour"], default="multicolour")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--spmv", choices=["auto", "csr", "sell", "sell2w", "sell4w"], default="auto",
                    help="single-RHS SpMV layout of the benchmark precision (auto: timed at the first solve)")
    ap.add_argument("--trsv", choices=["auto", "csr", "sell", "staged4", "staged12", "staged32", "packed12",
                                       "packed32", "split12", "split32"], default="auto",
                    help="single-RHS IC(0) sweep layout of the benchmark precision")
    ap.add_argument("--stop", choices=["residual", "estimate"], default="residual",
                    help="MINRES stop: ||b - Kx|| / ||b|| <= tol (the paper's relative residual) or |eta| / gamma_1")
    ap.add_argument("--pressure", choices=["diag", "pcg"], default="diag",
                    help="pressure block: Diag(Q_nu) or IC(0)-PCG on Q_nu (Sec. 6.4)")
    ap.add_argument("--k", type=int, default=1, help="right-hand sides per solve")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--inner-tol", type=float, default=1e-2)
    ap.add_argument("--no-variants", action="store_true")
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
    if not e or e.get("trsv") != trsv or e.get("precision") != precision:
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


def oracle_load(P, W):
    """The workload's load vector from the oracle (forcing seed 0)."""
    from paper_1309_5048_gb300.inputs import fourier_modes
    if W.get("load") == "cavity":
        return P.load_cavity()
    kappa, amp = fourier_modes(W["dim"], seed=0)
    return P.load_fourier(kappa, amp)


def cpu_baseline(W, ordering, tol, inner_tol, outer_full, target_s=15.0, pressure="diag", stop="residual"):
    """The oracle as it stands, single-threaded, on a bounded sample of one
    solve: the first m MINRES iterations, extrapolated to the full solve."""
    import numpy as np

    import oracle
    P = oracle.Problem(W["dim"], W["N"], W["p"], ordering=ordering)
    P.factor()
    P.factor_q()
    b = np.concatenate([oracle_load(P, W), np.zeros(P.n_p)])
    t = time.perf_counter()
    P.minres(b, tol=tol, inner_tol=inner_tol, max_outer=2, pressure=pressure, stop=stop)
    pilot = (time.perf_counter() - t) / 2
    m = int(max(2, min(outer_full, target_s / max(pilot, 1e-6))))
    t = time.perf_counter()
    _, info = P.minres(b, tol=tol, inner_tol=inner_tol, max_outer=m, pressure=pressure, stop=stop)
    dt = time.perf_counter() - t
    per_outer = dt / max(info["outer"], 1)
    est = per_outer * max(outer_full, 1)
    return {"value": 1.0 / est, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": "first %d of %d MINRES iterations of one solve (forcing seed 0), %.1f s, "
                      "extrapolated linearly to the full solve; oracle assembly/ordering/IC(0) excluded"
                      % (info["outer"], outer_full, dt)}


def run_reference(args):
    """--impl reference: the FP64 CPU oracle, each step a bounded sample."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    W = WORKLOADS[args.workload]
    P = oracle.Problem(W["dim"], W["N"], W["p"], ordering=args.ordering)
    P.factor()
    P.factor_q()
    b = np.concatenate([oracle_load(P, W), np.zeros(P.n_p)])
    pres = dict(pressure=args.pressure, stop=args.stop)
    # one untimed full solve gives the outer count used to extrapolate samples
    t = time.perf_counter()
    x, full = P.minres(b, tol=args.tol, inner_tol=args.inner_tol, **pres)
    t_full = time.perf_counter() - t
    outer_full = max(full["outer"], 1)
    per_outer_full = t_full / outer_full
    m = int(max(1, min(outer_full, 4.0 / max(per_outer_full, 1e-6))))  # ~4 s per step
    for _ in range(args.warmup):
        P.minres(b, tol=args.tol, inner_tol=args.inner_tol, max_outer=m, **pres)
    t = time.perf_counter()
    for _ in range(args.steps):
        _, info = P.minres(b, tol=args.tol, inner_tol=args.inner_tol, max_outer=m, **pres)
    dt = time.perf_counter() - t
    per_solve = dt / args.steps / max(info["outer"], 1) * outer_full
    value = 1.0 / per_solve
    sample = ("each step: first %d of %d MINRES iterations of one solve (seed 0), extrapolated; "
              "one untimed full solve took %.1f s" % (info["outer"], outer_full, t_full))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W["desc"], "ordering": args.ordering, "k": 1, "tol": args.tol,
                       "inner_tol": args.inner_tol,
                       "pressure_block": "Diag(Q)" if args.pressure == "diag" else "IC(0)-PCG(Q)",
                       "stop": args.stop},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "outer_its": outer_full, "relres_true": full["relres_true"]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = dist_env()
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
    W = WORKLOADS[args.workload]
    t0 = time.perf_counter()
    s = gb.Stokes(W["dim"], W["N"], W["p"], ordering=args.ordering)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    s.assemble(1.0)
    s.factor_ic0()
    if args.spmv != "auto" or args.trsv != "auto":
        s.set_kernel_variants(args.precision, args.spmv, args.trsv)
    torch.cuda.synchronize()
    t_rf = time.perf_counter() - t0
    k = args.k

    def make_rhs(k, seed0):
        rhs = torch.zeros(k, s.n, dtype=torch.float64, device="cuda")
        for t in range(k):
            if W.get("load") == "cavity":  # column t: lid speed 1 + t + seed0 / 1000
                rhs[t, : s.n_u] = s.load_cavity() * (1.0 + t + seed0 / 1000.0)
            else:
                kap, amp = fourier_modes(W["dim"], seed=seed0 + t)
                rhs[t, : s.n_u] = s.load_fourier(kap, amp)
        return rhs

    rhs = make_rhs(k, rank * 1000)
    out = torch.empty_like(rhs)
    opts = dict(tol=args.tol, inner_tol=args.inner_tol, precision=args.precision, use_graph=not args.no_graph,
                max_outer=args.max_outer, pressure=args.pressure, stop=args.stop)

    def timed(rhs_, out_, steps, warmup, **o):
        info = None
        for _ in range(warmup):
            _, info = s.solve(rhs_, out=out_, **o)
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            _, info = s.solve(rhs_, out=out_, **o)
        e1.record()
        torch.cuda.synchronize()
        barrier()
        return e0.elapsed_time(e1), info

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

    # end to end through the public host-buffer call (pinned memory)
    rhs_h = rhs.cpu().pin_memory()
    out_h = torch.empty_like(rhs_h).pin_memory()
    for _ in range(2):
        s.solve_host(rhs_h, out_h, **opts)
    barrier()
    t = time.perf_counter()
    for _ in range(args.steps):
        s.solve_host(rhs_h, out_h, **opts)
    e2e_s = max_over_ranks(time.perf_counter() - t, dist)
    bytes_io = 8 * k * s.n

    # per-kernel timing (events on the library's stream) and the roofline
    x_last = out.clone()
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
    roof = {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["gbs"], "peak": peak, "unit": "GB/s",
            "frac": kern[dom]["gbs"] / peak, "peak_source": peak_kind,
            "traffic": traffic_for(dom, args.workload, s.kernel_variants(args.precision)[1], args.precision),
            "unit_of_launch": ("one preconditioner application: forward + backward IC(0) sweep over %d levels "
                               "each" % s.nlevels) if dom == "ic0_apply" else "one kernel launch"}
    del x_last
    # the whole solve against the same peak: algorithmic bytes from the
    # measured counts over the measured time per solve (k = 1, Diag(Q) only)
    whole = None
    if k == 1 and args.pressure == "diag":
        sb = solve_bytes(s, infos[0], args.precision)
        gbs = sb / (ms / args.steps * 1e-3) / 1e9
        whole = {"bytes_per_solve": sb, "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                 "peak_source": peak_kind}

    variants = {}
    if not args.no_variants and rank == 0:
        # Diag(Q_nu) pressure block (the configuration above) in other
        # precisions / batch widths, and the paper's IC(0)-PCG(A,Q) block
        for name, prec, kk, pres in (("mixed_k1", "mixed", 1, "diag"), ("fp64_k32", "fp64", 32, "diag"),
                                     ("mixed_k32", "mixed", 32, "diag"), ("fp64_k1_pcgq", "fp64", 1, "pcg"),
                                     ("mixed_k1_pcgq", "mixed", 1, "pcg"), ("mixed_k32_pcgq", "mixed", 32, "pcg")):
            r = make_rhs(kk, 5000)
            o = torch.empty_like(r)
            st = 1 if kk > 1 else max(1, args.steps // 2)
            ms_v, inf_v = timed(r, o, st, 1, tol=args.tol, inner_tol=args.inner_tol, precision=prec,
                                use_graph=not args.no_graph, pressure=pres, stop=args.stop)
            iv = inf_v if isinstance(inf_v, list) else [inf_v]
            variants[name] = {"solves_per_s": st * kk / (ms_v / 1000.0), "k": kk, "precision": prec,
                              "pressure_block": "Diag(Q)" if pres == "diag" else "IC(0)-PCG(Q)",
                              "outer_its_mean": statistics.mean(i["outer_its"] for i in iv),
                              "inner_its_mean": statistics.mean(i["inner_its_total"] for i in iv),
                              "relres_true_max": max(i["relres_true"] for i in iv)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(W, args.ordering, args.tol, args.inner_tol, int(infos[0]["outer_its"]),
                           pressure=args.pressure, stop=args.stop)

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
            "e2e": {"value": throughput(world, args.steps, k, 1000.0 * e2e_s), "unit": "solves/s",
                    "h2d_bytes_per_step": bytes_io,
                    "d2h_bytes_per_step": bytes_io},
            "gpu_launches": int(args.steps * sum(launches_per_solve(s, i, args.pressure) for i in infos)),
            "clocks": clock_info,
            "outer_its": infos[0]["outer_its"], "inner_its_total": infos[0]["inner_its_total"],
            "inner_its_mean": infos[0]["inner_its_total"] / max(infos[0]["precond_apps"], 1),
            "relres_est": infos[0]["relres_est"], "relres_true": infos[0]["relres_true"],
            "setup_s": t_setup, "assemble_factor_s": t_rf, "levels": s.nlevels,
            "layouts": dict(zip(("spmv", "trsv"), s.kernel_variants(args.precision))),
            "kernels": kern, "variants": variants,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
