#!/usr/bin/env python
"""Benchmark: assembled entries/s and solves/s of the weighted-quadrature
IgA-SGBEM path on the precision workload (the star r = 0.4(1 + 0.2 cos 5 theta)
as a 256-point periodic cubic, n = 16384 DoF, degree 4, N_ref = 2,
u = log|x - (2,1)|).

One step = one request through the whole path on the device: geometry at the
nodes, fused assembly of A, right-hand side, Cholesky factorisation and solve
(MIXED tier: FP32 assembly far field, tensor-core factor on a three-term
FP16 split with FP32 accumulation, float-float iterative refinement to
1e-10).  Rules are built once per discretisation
(untimed) and reused, as a serving process does.  The same line carries the
plain FP64 GPU form of the same request, the n = 2048, p = 3 request, a short
run of the served workload, the measured pipe peaks the roofline fractions
divide by, and the CPU oracle on a bounded sample.

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# DRAM read + write bytes of one launch of the FP32 assembly kernel, keyed by
# (n, degree, N_ref): ncu captures summarised in profiles/ (the file named in
# the value); a configuration without a capture of the current kernel gets null
ASSEMBLY_TRAFFIC = {(16384, 4, 2): (86.26e6 + 2.09e9, "profiles/ncu_assemble_f_traffic_star16384_star2048.md"),
                    (2048, 3, 2): (8.46e6 + 15.1e3, "profiles/ncu_assemble_f_traffic_star16384_star2048.md")}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--degree", type=int, default=4)
    ap.add_argument("--nref", type=int, default=2)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--fp64-warmup", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the n = 2048 request and the short served-workload run")
    ap.add_argument("--workload", choices=["request", "batch", "serve"], default="request",
                    help="request: one assemble+rhs+solve request per step (default); batch: 1024 uneven "
                         "assemblies per step; serve: Poisson arrivals through the request server")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-seconds", type=float, default=0.5)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=float, default=180.0)
    ap.add_argument("--serve-distinct", type=int, default=0,
                    help="draw every request from a pool of this many (curve, n, p) problems (0: all distinct)")
    ap.add_argument("--serve-cache-gb", type=float, default=16.0,
                    help="device memory the server keeps for resident problems (rules, matrix, factor)")
    ap.add_argument("--serve-fp64-sample", type=int, default=8)
    ap.add_argument("--batch-count", type=int, default=1024)
    ap.add_argument("--fp64-sample", type=int, default=64)
    ap.add_argument("--cpu-rows-per-core", type=int, default=2)
    return ap.parse_args()


def measured_peak(key: str, fallback: float) -> tuple[float, str]:
    """A peak from MEASURED_PEAKS.json at the repository root (measured copy
    bandwidth and GEMM throughput of this GPU model), else the stated fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)[key]), "measured"
    except (OSError, KeyError, ValueError):
        return fallback, "fallback"


def all_reduce_value(x: float, op: str = "max") -> float:
    """Max or sum of a per-rank number over the ranks of the job (the number
    itself when the job has one rank); NCCL jobs reduce on the device, gloo
    jobs on the host."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampled every 200 ms during the timed region."""
    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


# --------------------------------------------------------------------------- measured pipe peaks
def measure_pipes(igs, ctx, device: int) -> dict:
    """FP32 FMA, MUFU lg2 / rcp and FP64 FMA throughput of this GPU by the
    library's probe kernels (CUDA events), with the SM clock sampled while
    they run."""
    clk = ClockSampler(device)
    clk.start()
    out = {}
    for key, kind, unit in (("fp32_fma", igs.IGS_PEAK_FP32_FMA, "TFLOP/s"), ("mufu_lg2", igs.IGS_PEAK_MUFU_LG2, "Tops/s"),
                            ("mufu_rcp", igs.IGS_PEAK_MUFU_RCP, "Tops/s"), ("fp64_fma", igs.IGS_PEAK_FP64_FMA, "TFLOP/s")):
        best, ms = 0.0, None
        for _ in range(3):
            rate, t = igs.igs_measure_peak(ctx, kind)
            if rate > best:
                best, ms = rate, t
        out[key] = {"value": best / 1e12, "unit": unit, "ms": ms}
    out["clocks"] = clk.stop()
    out["how"] = ("igs_measure_peak: every SM filled with 8 independent chains per thread of one instruction "
                  "kind, best of 3 launches timed with CUDA events")
    return out


def assembly_work(nq: int, n: int, d: int) -> dict:
    """Algorithmic work of one assembly (the method's count, Sect. 5.1 cost
    model): N_quad(N_quad+1)/2 evaluations of the symmetric K1 (one log, one
    reciprocal and 12 flop each, log and reciprocal counted as one flop),
    2(d+1) flop of K1 contraction and 2(d+1) of W^s Q per ordered node pair,
    and 2 N_quad n (d+1) flop of the second contraction."""
    unique = nq * (nq + 1) // 2
    ordered = nq * nq
    flop = 14 * unique + 4 * (d + 1) * ordered + 2 * nq * n * (d + 1)
    return {"flop": flop, "k1_unique_evaluations": unique, "k1_evaluated": ordered,
            "mufu_ops": 2 * unique, "mufu_evaluated": 2 * ordered}


# --------------------------------------------------------------------------- one request per step
def request_run(igs, ctx, geom, data, n, d, nref, tier, steps, warmup, flush, stream, world, clocks_dev=None):
    """Warm-up, then `steps` timed requests (assemble, then right-hand side
    beside the factorisation, then the solve) on one problem; device times by
    CUDA events on the context stream, L2 flushed between steps outside them."""
    import torch
    dev = flush.device
    prob = igs.igs_create_problem(geom, d, n, nref, tier)
    igs.igs_build_weighted_rules(prob)
    xy = igs.igs_rhs_points(prob)
    uD = torch.tensor(data.value(xy[:, 0], xy[:, 1])[None, :], dtype=torch.float64, device=dev)
    alpha = torch.empty((1, n), dtype=torch.float64, device=dev)

    def step(times, launches, phases):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        igs.igs_assemble(prob)
        t = igs.igs_problem_timing(prob)
        ph = {"geometry": t.geometry_ms, "assemble": t.assemble_ms}
        nl = t.kernel_launches
        _, res = igs.igs_solve_data(prob, uD, alpha)
        t = igs.igs_problem_timing(prob)
        ph["rhs"], ph["factor"], ph["solve"] = t.rhs_ms, t.factor_ms, t.solve_ms
        nl += t.kernel_launches
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
        launches.append(nl)
        phases.append(ph)
        flush.zero_()                       # evict L2 between steps (outside the timed events)
        torch.cuda.synchronize()
        return res[0], t.ir_iterations

    scratch = ([], [], [])
    for _ in range(warmup):
        step(*scratch)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(clocks_dev) if clocks_dev is not None else None
    if clk:
        clk.start()
    times, launches, phases = [], [], []
    wall0 = time.perf_counter()
    last = None
    for _ in range(steps):
        last = step(times, launches, phases)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    ck = clk.stop() if clk else None
    total_ms = all_reduce_value(sum(times), "max")         # slowest rank sets the job time
    ts = sorted(times)
    return dict(prob=prob, uD=uD, times=times, total_ms=total_ms, wall=wall, launches=launches, phases=phases,
                resid=last[0], ir=last[1], clocks=ck, steps=steps,
                ms_per_step=total_ms / steps,
                p50=ts[len(ts) // 2], p99=ts[min(len(ts) - 1, int(math.ceil(0.99 * len(ts))) - 1)],
                phase_mean={k: statistics.mean(p[k] for p in phases) for k in phases[0]})


def band_errors(A32, A64, n: int, d: int) -> dict:
    """Relative Frobenius error of the MIXED matrix per entry band (cyclic
    distance |i - j| <= d+1, <= 8(d+1), farther), by row blocks."""
    import torch
    bands = (("near(|i-j|<=d+1)", 0, d + 1), ("mid(<=8(d+1))", d + 2, 8 * (d + 1)), ("far", 8 * (d + 1) + 1, n))
    num = {b[0]: 0.0 for b in bands}
    den = {b[0]: 0.0 for b in bands}
    col = torch.arange(n, device=A64.device)
    for r0 in range(0, n, 1024):
        r1 = min(n, r0 + 1024)
        row = torch.arange(r0, r1, device=A64.device)
        dist = (row[:, None] - col[None, :]).abs()
        dist = torch.minimum(dist, n - dist)
        E = (A32[r0:r1] - A64[r0:r1]) ** 2
        R = A64[r0:r1] ** 2
        for label, lo, hi in bands:
            m = (dist >= lo) & (dist <= hi)
            num[label] += float(E[m].sum())
            den[label] += float(R[m].sum())
    return {k: math.sqrt(num[k] / den[k]) if den[k] > 0 else None for k in num}


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1703_10016_gb300 import build as build_mod
    build_mod.build_library()
    from paper_1703_10016_gb300 import igs
    from paper_1703_10016_gb300 import workloads as wl

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    n, d, nref = args.n, args.degree, args.nref
    curve = wl.star_curve()
    data = wl.Harmonic("log", (2.0, 1.0))
    ctx = igs.igs_create(local_rank, stream.cuda_stream)
    geom = igs.igs_create_geometry(ctx, curve.degree, curve.knots, curve.ctrl, curve.weights, curve.closed)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2

    peaks = measure_pipes(igs, ctx, local_rank)
    mixed = request_run(igs, ctx, geom, data, n, d, nref, igs.IGS_MIXED, args.steps, args.warmup, flush, stream,
                        world, clocks_dev=local_rank)
    fp = request_run(igs, ctx, geom, data, n, d, nref, igs.IGS_FP64, max(args.fp64_steps, 1), args.fp64_warmup,
                     flush, stream, world)
    A32 = torch.empty((n, n), dtype=torch.float64, device=dev)
    A64 = torch.empty((n, n), dtype=torch.float64, device=dev)
    igs.igs_get_matrix(mixed["prob"], A32)
    igs.igs_get_matrix(fp["prob"], A64)
    rel_err = float(torch.linalg.norm(A32 - A64) / torch.linalg.norm(A64))
    # the discrete operator is symmetric only up to the quadrature error (A is used as (A + A^T)/2)
    asym = {k: float(torch.linalg.norm(M - M.T) / torch.linalg.norm(M)) for k, M in (("mixed", A32), ("fp64", A64))}
    bands = band_errors(A32, A64, n, d)
    del A32, A64
    torch.cuda.empty_cache()

    # ------------------------------------------------------------------ roofline (assembly kernel)
    info = igs.igs_problem_info(mixed["prob"])
    nq = info.n_quad
    work = assembly_work(nq, n, d)
    asm_ms = mixed["phase_mean"]["assemble"]                # CUDA events around the one assembly launch
    achieved = work["flop"] / (asm_ms * 1e-3) / 1e12
    fp32_peak = peaks["fp32_fma"]["value"]
    mufu_peak = peaks["mufu_lg2"]["value"]
    traffic = ASSEMBLY_TRAFFIC.get((n, d, nref))
    step_ms = mixed["ms_per_step"]
    value = world * n * n * mixed["steps"] / (mixed["total_ms"] * 1e-3)
    fp_step = fp["ms_per_step"]
    fac_ms = mixed["phase_mean"]["factor"]
    f16_peak, f16_src = measured_peak("bf16_tflops_sustained", 1700.0)   # kind::f16 runs FP16 at the BF16 rate

    out = {
        "metric": "assembled entries/s (assemble + rhs + solve per request, MIXED tier, <=1e-6 rel. error)",
        "value": value,
        "unit": "entries/s",
        "n_gpus": world,
        "steps": mixed["steps"],
        "warmup": args.warmup,
        "ms_per_step": step_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": f"star256 r=0.4(1+0.2cos5t), n={n}, p={d}, N_ref={nref}, u=log|x-(2,1)|, 1 rhs",
                   "n": n, "degree": d, "n_ref": nref, "n_quad": nq, "parallelism": f"replicas x{world}",
                   "l2": "256 MB flush between timed steps (outside the step events); A is larger than L2"},
        "solves_per_s": world * mixed["steps"] / (mixed["total_ms"] * 1e-3),
        "p50_ms": mixed["p50"],
        "p99_ms": mixed["p99"],
        "phases_ms": mixed["phase_mean"],
        "phases_note": "rhs runs on a second stream beside factor (igs_solve_data): the phases overlap",
        "dominant_phase": max(mixed["phase_mean"], key=mixed["phase_mean"].get),
        "rel_err_vs_fp64": rel_err,
        "rel_err_vs_fp64_by_band": bands,
        "asymmetry_rel_frobenius": asym,
        "ir_iterations": mixed["ir"],
        "final_residual": mixed["resid"],
        "fp64": {"value": world * n * n * fp["steps"] / (fp["total_ms"] * 1e-3), "unit": "entries/s",
                 "ms_per_step": fp_step, "solves_per_s": world * fp["steps"] / (fp["total_ms"] * 1e-3),
                 "phases_ms": fp["phase_mean"], "steps": fp["steps"], "warmup": args.fp64_warmup},
        "speedup_mixed_vs_fp64": fp_step / step_ms,
        "roofline": {"kernel": f"k_assemble_f<{d},{'true' if curve.closed else 'false'}>", "bound": "alu",
                     "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": traffic[0] if traffic else None,
                     "traffic_source": traffic[1] if traffic else "no capture of the current kernel at this size",
                     "work": work,
                     "work_rule": "14 flop per unique K1 evaluation N_quad(N_quad+1)/2 + 4(d+1) per ordered node "
                                  "pair (K1 and W^s Q contractions) + 2 N_quad n (d+1)",
                     "peak_basis": "measured FP32 FMA throughput (igs_measure_peak), of measured",
                     "launch_ms": asm_ms,
                     "mufu": {"achieved": work["mufu_ops"] / (asm_ms * 1e-3) / 1e12, "peak": mufu_peak,
                              "unit": "Tops/s", "frac": work["mufu_ops"] / (asm_ms * 1e-3) / 1e12 / mufu_peak,
                              "evaluated_frac": work["mufu_evaluated"] / (asm_ms * 1e-3) / 1e12 / mufu_peak,
                              "note": "one log and one reciprocal per unique K1 evaluation; the kernel evaluates "
                                      "both (a,b) and (b,a), twice the method's count (evaluated_frac)",
                              "peak_basis": "measured lg2.approx throughput, of measured"}},
        "factor_rate": {"flop": n ** 3 / 3, "achieved_tflops": n ** 3 / 3 / (fac_ms * 1e-3) / 1e12,
                        "mma_issue_tflops": n ** 3 / (fac_ms * 1e-3) / 1e12,
                        "f16_peak_tflops": f16_peak, "peak_source": f"{f16_src} bf16 sustained (FP16 dense rate)",
                        "frac": n ** 3 / 3 / (fac_ms * 1e-3) / 1e12 / f16_peak,
                        "note": "the three-term FP16 split (hi.hi + hi.lo + lo.hi) issues three MMAs per product "
                                "(mma_issue_tflops); the SIMT panel chain runs beside the tensor-core update; "
                                "phase time overlaps the rhs"},
        "measured_peaks": peaks,
        "gpu_launches": int(sum(mixed["launches"])),
        "clocks": mixed["clocks"],
    }

    # ------------------------------------------------------------------ e2e through host buffers
    if not args.no_e2e:
        prob = mixed["prob"]
        e2e_times, h2d, d2h = [], 0, 0
        for it in range(args.warmup + mixed["steps"]):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g2 = igs.igs_create_geometry(ctx, curve.degree, curve.knots, curve.ctrl, curve.weights, curve.closed)
            igs.igs_set_geometry(prob, g2)
            xy = igs.igs_rhs_points(prob)
            igs.igs_assemble(prob)                       # queued: the host evaluates u_D meanwhile
            u = data.value(xy[:, 0], xy[:, 1])[None, :]
            alpha, res = igs.igs_solve_data(prob, u)
            t1 = time.perf_counter()
            igs.igs_set_geometry(prob, geom)
            igs.igs_destroy_geometry(g2)
            if it >= args.warmup:
                e2e_times.append(t1 - t0)
            h2d = 8 * (len(curve.knots) + curve.ctrl.size + (len(curve.ctrl) if curve.weights is not None else 0)) + 8 * u.size
            d2h = 8 * xy.size + 8 * alpha.size
        e2e_total = all_reduce_value(sum(e2e_times), "max")
        out["e2e"] = {"value": world * n * n * len(e2e_times) / e2e_total, "unit": "entries/s",
                      "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                      "ms_per_step": 1e3 * e2e_total / len(e2e_times),
                      "includes": "new geometry upload, rhs points D2H, assemble (host u_D beside it), rhs upload, solve, alpha D2H"}
    for r in (mixed, fp):
        igs.igs_destroy_problem(r["prob"])

    # ------------------------------------------------------------------ n = 2048 request, short served run
    if not args.no_extras:
        c2 = request_run(igs, ctx, geom, data, 2048, 3, 2, igs.IGS_MIXED, 20, 3, flush, stream, world)
        igs.igs_destroy_problem(c2["prob"])
        w2 = assembly_work(igs_n_quad(2048, 3, 2), 2048, 3)
        a2 = c2["phase_mean"]["assemble"]
        out["star2048_p3"] = {"value": world * 2048 ** 2 * c2["steps"] / (c2["total_ms"] * 1e-3), "unit": "entries/s",
                              "ms_per_step": c2["ms_per_step"], "p50_ms": c2["p50"], "p99_ms": c2["p99"],
                              "phases_ms": c2["phase_mean"], "steps": c2["steps"], "ir_iterations": c2["ir"],
                              "assembly_frac_of_fp32_peak": w2["flop"] / (a2 * 1e-3) / 1e12 / fp32_peak}
    igs.igs_destroy_geometry(geom)
    igs.igs_destroy(ctx)
    del flush
    torch.cuda.empty_cache()
    if not args.no_extras:
        sv = serve_workload(igs, wl, local_rank, world, rate=2000.0, seconds=0.25, slots=args.serve_slots,
                            budget_gb=args.serve_budget_gb, cache_gb=args.serve_cache_gb, distinct=0, warmup=2,
                            fp64_sample=4)
        out["served_2000rps_0.25s"] = {k: sv[k] for k in ("value", "unit", "requests", "completed", "failed",
                                                           "latency_ms", "queue_ms", "run_ms", "serial_fp64_loop",
                                                           "speedup_vs_serial_fp64", "entries_per_s")}

    # ------------------------------------------------------------------ CPU oracle baseline
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(n, d, nref, args.cpu_rows_per_core)
    return out


def igs_n_quad(n: int, d: int, nref: int) -> int:
    """N_quad = 2d + 2 N_ref n - 1 for a closed curve (Sect. 4)."""
    return 2 * d + 2 * nref * n - 1

# --------------------------------------------------------------------------- batched form
def run_batch(args, rank, world, local_rank):
    """Batched workload: `batch_count` random stars (n log-uniform in [64, 4096],
    p in {2, 3, 4}, N_ref = 2) assembled per step by one persistent launch."""
    import torch
    from paper_1703_10016_gb300 import build as build_mod
    build_mod.build_library()
    from paper_1703_10016_gb300 import igs
    from paper_1703_10016_gb300 import workloads as wl
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    ctx = igs.igs_create(local_rank, stream.cuda_stream)
    peaks = measure_pipes(igs, ctx, local_rank)
    mix = wl.batch_mix(args.batch_count, seed=4)
    t0 = time.perf_counter()
    geoms, probs = [], []
    for pr in mix:
        c = pr.curve
        g = igs.igs_create_geometry(ctx, c.degree, c.knots, c.ctrl, c.weights, c.closed)
        p = igs.igs_create_problem(g, pr.degree, pr.n_elems, pr.n_ref, igs.IGS_MIXED)
        igs.igs_build_weighted_rules(p)
        geoms.append(g)
        probs.append(p)
    rules_s = time.perf_counter() - t0
    entries = sum(pr.n_elems * pr.n_elems for pr in mix)
    nq = [igs.igs_problem_info(p).n_quad for p in probs]
    b = igs.igs_batch_create(ctx, probs)
    igs.igs_batch_assemble(b)
    best = igs.igs_batch_tune(b, reps=1)
    for _ in range(args.warmup):
        igs.igs_batch_assemble(b)
    clk = ClockSampler(local_rank)
    clk.start()
    times = [igs.igs_batch_assemble(b) for _ in range(args.steps)]
    clocks = clk.stop()
    step_ms = all_reduce_value(statistics.mean(times), "max")
    # single-problem loop, MIXED (same kernels one launch per problem)
    torch.cuda.synchronize()
    loop_ms = 0.0
    for p in probs:
        igs.igs_assemble(p)
        tm = igs.igs_problem_timing(p)
        loop_ms += tm.geometry_ms + tm.assemble_ms
    # plain FP64 GPU form on a seeded sample, and the MIXED error against it
    rng = __import__("numpy").random.default_rng(7)
    sample = sorted(rng.choice(len(mix), size=min(args.fp64_sample, len(mix)), replace=False).tolist())
    fp_ms, fp_entries, errs = 0.0, 0, []
    for k in sample:
        pr = mix[k]
        p64 = igs.igs_create_problem(geoms[k], pr.degree, pr.n_elems, pr.n_ref, igs.IGS_FP64)
        A64 = torch.empty((pr.n_elems, pr.n_elems), dtype=torch.float64, device="cuda")
        igs.igs_assemble(p64, A64)
        tm = igs.igs_problem_timing(p64)
        fp_ms += tm.geometry_ms + tm.assemble_ms
        fp_entries += pr.n_elems * pr.n_elems
        A32 = torch.empty((pr.n_elems, pr.n_elems), dtype=torch.float64, device="cuda")
        igs.igs_get_matrix(probs[k], A32)
        errs.append(float(torch.linalg.norm(A32 - A64) / torch.linalg.norm(A64)))
        igs.igs_destroy_problem(p64)
    pairs = sum(q * q for q in nq)
    flops = sum(assembly_work(q, pr.n_elems, pr.degree)["flop"] for q, pr in zip(nq, mix))
    achieved = flops / (step_ms * 1e-3) / 1e12
    peak = peaks["fp32_fma"]["value"]
    out = {
        "metric": "assembled entries/s (batched assembly, MIXED tier, <=1e-6 rel. error)",
        "value": world * entries / (step_ms * 1e-3), "unit": "entries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"batch{len(mix)} random stars r=0.4(1+sum a_k cos(k t+phi_k)), n log-uniform "
                               f"[64,4096], p in {{2,3,4}}, N_ref=2 (seed 4)",
                   "entries_per_step": entries, "node_pairs_per_step": pairs, "parallelism": f"replicas x{world}",
                   "l2": "inputs and outputs (A: %.1f GB FP32) larger than L2" % (4 * entries / 1e9)},
        "tuned": best,
        "rules_setup_s": rules_s,
        "single_problem_loop_mixed": {"value": entries / (loop_ms * 1e-3), "unit": "entries/s",
                                      "ms": loop_ms, "launches": 3 * len(mix)},
        "fp64_loop_sample": {"value": fp_entries / (fp_ms * 1e-3), "unit": "entries/s", "problems": len(sample),
                             "entries": fp_entries, "ms": fp_ms},
        "speedup_vs_fp64_loop": (entries / (step_ms * 1e-3)) / (fp_entries / (fp_ms * 1e-3)),
        "rel_err_vs_fp64_max": max(errs), "rel_err_vs_fp64_median": statistics.median(errs),
        "roofline": {"kernel": "k_batch_assemble_f", "bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                     "work": "per problem: 14 flop per unique K1 evaluation + 4(p+1) per ordered node pair "
                             "+ 2 n_quad n (p+1)",
                     "peak_basis": "measured FP32 FMA throughput (igs_measure_peak), of measured"},
        "measured_peaks": peaks,
        "gpu_launches": 2,
        "clocks": clocks,
    }
    igs.igs_batch_destroy(b)
    for p in probs:
        igs.igs_destroy_problem(p)
    for g in geoms:
        igs.igs_destroy_geometry(g)
    igs.igs_destroy(ctx)
    return out


# --------------------------------------------------------------------------- served form
def _serve_data(xy, k):
    import numpy as np
    src = [2.5 * np.array([np.cos(2 * np.pi * j / 8), np.sin(2 * np.pi * j / 8)]) for j in range(k)]
    return np.stack([np.log(np.hypot(xy[:, 0] - s[0], xy[:, 1] - s[1])) for s in src])


def serve_workload(igs, wl, local_rank, world, rate, seconds, slots, budget_gb, cache_gb, distinct, warmup,
                   fp64_sample):
    """Served workload: Poisson arrivals (seed 5) of assemble+solve requests, random
    stars, n log-uniform in [128, 16384], p in {2, 3, 4}, 1..8 data sets each,
    through the request server (memory admission), against a serial FP64 loop."""
    import numpy as np
    import torch
    torch.cuda.set_device(local_rank)
    arrivals = wl.serve_arrivals(rate, seconds, seed=5)
    if distinct > 0:
        # a recurring workload: the same problems come back with new data
        pool = [pr for _, pr, _ in arrivals[:distinct]]
        pick = np.random.default_rng(6).integers(0, len(pool), size=len(arrivals))
        arrivals = [(ta, pool[k], nrhs) for (ta, _, nrhs), k in zip(arrivals, pick)]
    srv = igs.igs_server_create(local_rank, slots=slots, mem_budget=int(budget_gb * 1e9),
                                cache_budget=int(cache_gb * 1e9))
    # warm-up: a few small requests (module loading, first graph builds)
    warm = [igs.igs_server_submit(srv, wl.star_curve(), 3, 128, 2, igs.IGS_MIXED, 1, _serve_data)
            for _ in range(max(1, warmup))]
    igs.igs_server_drain(srv)
    for t in warm:
        st = igs.igs_server_wait(srv, t)
        igs.igs_server_result(srv, t, st["n"], 1)
    clk = ClockSampler(local_rank)
    clk.start()
    t0 = time.perf_counter()
    tickets = []
    for (ta, pr, nrhs) in arrivals:
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        tickets.append((igs.igs_server_submit(srv, pr.curve, pr.degree, pr.n_elems, pr.n_ref, igs.IGS_MIXED, nrhs,
                                              _serve_data), pr, nrhs))
    igs.igs_server_drain(srv)
    wall = time.perf_counter() - t0
    clocks = clk.stop()
    lat, queue, run, fails, entries, solves, bytes_max = [], [], [], 0, 0, 0, 0
    reuse = {"rules": 0, "factor": 0}
    fail_kinds = {}
    for t, pr, nrhs in tickets:
        st = igs.igs_server_wait(srv, t)
        if st["status"] != igs.IGS_REQ_DONE:
            fails += 1
            try:
                igs.igs_server_result(srv, t, max(st["n"], 1), nrhs)
            except igs.IgsError as e:
                key = f"{e.code}: {str(e).split(': ', 1)[-1][:120]} (n={pr.n_elems}, p={pr.degree})"
                fail_kinds[key] = fail_kinds.get(key, 0) + 1
            continue
        _, res, st = igs.igs_server_result(srv, t, st["n"], nrhs)
        if st["reuse"] == igs.IGS_REUSE_RULES:
            reuse["rules"] += 1
        elif st["reuse"] == igs.IGS_REUSE_FACTOR:
            reuse["factor"] += 1
        lat.append(st["latency_ms"])
        queue.append(st["queue_ms"])
        run.append(st["run_ms"])
        entries += st["n"] ** 2
        solves += 1
        bytes_max = max(bytes_max, st["device_bytes"])
    igs.igs_server_destroy(srv)
    lat_s = sorted(lat)
    pct = lambda q: lat_s[min(len(lat_s) - 1, int(math.ceil(q * len(lat_s))) - 1)] if lat_s else None
    # whole job: every rank serves its own replica of the arrival stream
    job_wall = all_reduce_value(wall, "max")
    job_solves = all_reduce_value(solves, "sum")
    job_entries = all_reduce_value(entries, "sum")
    # serial FP64 loop on a seeded sample of the same requests (direct API, one at a time)
    rng = np.random.default_rng(9)
    sample = sorted(rng.choice(len(arrivals), size=min(fp64_sample, len(arrivals)), replace=False).tolist())
    ctx = igs.igs_create(local_rank)
    fp_ms, fp_entries = 0.0, 0
    for k in sample:
        _, pr, nrhs = arrivals[k]
        c = pr.curve
        g = igs.igs_create_geometry(ctx, c.degree, c.knots, c.ctrl, c.weights, c.closed)
        p = igs.igs_create_problem(g, pr.degree, pr.n_elems, pr.n_ref, igs.IGS_FP64)
        torch.cuda.synchronize()
        ts = time.perf_counter()
        igs.igs_build_weighted_rules(p)
        igs.igs_assemble(p)
        xy = igs.igs_rhs_points(p)
        igs.igs_build_rhs(p, _serve_data(xy, nrhs))
        igs.igs_solve(p, nrhs=nrhs)
        fp_ms += 1e3 * (time.perf_counter() - ts)
        fp_entries += pr.n_elems ** 2
        igs.igs_destroy_problem(p)
        igs.igs_destroy_geometry(g)
    igs.igs_destroy(ctx)
    fp_rate = len(sample) / (fp_ms * 1e-3)
    return {
        "metric": "solves/s (served assemble+solve requests, MIXED tier, <=1e-6 rel. error)",
        "value": job_solves / job_wall, "unit": "solves/s", "n_gpus": world, "steps": len(tickets),
        "warmup": len(warm), "ms_per_step": 1e3 * wall / max(len(tickets), 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"Poisson {rate:g} req/s for {seconds:g} s (seed 5): random "
                               "stars, n log-uniform [128,16384], p in {2,3,4}, N_ref=2, 1..8 data sets"
                               + (f"; drawn from {distinct} recurring problems" if distinct else ""),
                   "slots": slots, "mem_budget_gb": budget_gb,
                   "resident_cache_gb": cache_gb,
                   "parallelism": f"replicas x{world}"},
        "requests": len(tickets), "completed": solves, "failed": fails, "reused": reuse, "failures": dict(list(fail_kinds.items())[:8]),
        "wall_s": wall,
        "offered_rate": rate, "achieved_rate": solves / wall,
        "latency_ms": {"p50": pct(0.5), "p99": pct(0.99), "mean": statistics.mean(lat) if lat else None},
        "queue_ms": {"p50": statistics.median(queue) if queue else None, "max": max(queue) if queue else None},
        "run_ms": {"p50": statistics.median(run) if run else None, "max": max(run) if run else None},
        "entries_per_s": job_entries / job_wall, "max_request_bytes": bytes_max,
        "serial_fp64_loop": {"value": fp_rate, "unit": "solves/s", "sample": len(sample), "ms": fp_ms,
                             "entries_per_s": fp_entries / (fp_ms * 1e-3)},
        "speedup_vs_serial_fp64": (solves / wall) / fp_rate,
        "gpu_launches": None,
        "clocks": clocks,
    }


def run_serve(args, rank, world, local_rank):
    from paper_1703_10016_gb300 import build as build_mod
    build_mod.build_library()
    from paper_1703_10016_gb300 import igs
    from paper_1703_10016_gb300 import workloads as wl
    return serve_workload(igs, wl, local_rank, world, args.serve_rate, args.serve_seconds, args.serve_slots,
                          args.serve_budget_gb, args.serve_cache_gb, args.serve_distinct, args.warmup,
                          args.serve_fp64_sample)


# --------------------------------------------------------------------------- CPU oracle (baseline and reference arm)
def _oracle_rules_chunk(job):
    """Regular rules of test functions lo..hi-1 (a pool task)."""
    from oracle.assembly import make_discretization
    from oracle.sampled import regular_rules_sparse
    from paper_1703_10016_gb300 import workloads as wl
    n, d, nref, lo, hi = job
    return regular_rules_sparse(make_discretization(wl.star_curve(), n, d, nref), range(lo, hi))


_ORACLE_ROWS = None


def _oracle_init(n, d, nref, rules):
    global _ORACLE_ROWS
    from oracle.sampled import RowSampler
    from paper_1703_10016_gb300 import workloads as wl
    _ORACLE_ROWS = RowSampler(wl.star_curve(), n, d, nref, rules=rules)


def _oracle_row(i):
    t0 = time.perf_counter()
    r = _ORACLE_ROWS.row(int(i))
    return float(r[int(i)]), time.perf_counter() - t0


def oracle_rows_timed(n, d, nref, row_sets, cores):
    """The oracle (plain FP64 numpy, oracle.sampled.RowSampler) on `cores`
    single-threaded worker processes (spawn): the rules of Algorithm 1 are
    built once, untimed; then each set of rows is computed across the pool
    and its wall time taken.  Returns (setup_s, [seconds per set])."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    step = max(1, (n + 4 * cores - 1) // (4 * cores))
    with ctx.Pool(cores) as pool:
        parts = pool.map(_oracle_rules_chunk, [(n, d, nref, lo, min(n, lo + step)) for lo in range(0, n, step)])
    rules = [x for p in parts for x in p]
    times = []
    with ctx.Pool(cores, initializer=_oracle_init, initargs=(n, d, nref, rules)) as pool:
        pool.map(_oracle_row, list(range(cores)))            # every worker set up before timing
        setup = time.perf_counter() - t0
        for rows in row_sets:
            t1 = time.perf_counter()
            pool.map(_oracle_row, list(rows), chunksize=1)
            times.append(time.perf_counter() - t1)
    return setup, times


ORACLE_RUNNER = """
import json, sys
sys.path.insert(0, {root!r})
import bench
setup, times = bench.oracle_rows_timed({n}, {d}, {nref}, {row_sets!r}, {cores})
print(json.dumps({{"setup_s": setup, "times": times}}))
"""


def host_cpu() -> dict:
    """Host core count and CPU model (lscpu, else /proc/cpuinfo, else platform)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "model": model or platform.processor() or platform.machine(),
            "machine": platform.machine()}


def run_oracle(n, d, nref, row_sets, cores, timeout=1200):
    """oracle_rows_timed in a fresh interpreter (its spawn pool starts before
    any GPU call of that process), one BLAS thread per worker."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_RUNNER.format(root=ROOT, n=n, d=d, nref=nref, row_sets=[list(r) for r in row_sets], cores=cores)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-400:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(n, d, nref, rows_per_core=2):
    """The oracle on all host cores, a bounded sample: rows_per_core full rows
    of A per core (rows spread over the matrix)."""
    cpu = host_cpu()
    cores = max(1, cpu["nproc"] or 1)
    k = rows_per_core * cores
    rows = [(q * 7919) % n for q in range(k)]
    try:
        res = run_oracle(n, d, nref, [rows], cores)
    except (RuntimeError, subprocess.SubprocessError) as e:
        return {"value": None, "unit": "entries/s", "cores": cores, "kind": "oracle", "sample": f"failed: {e}"}
    sec = res["times"][0]
    return {"value": k * n / sec, "unit": "entries/s", "cores": cores, "kind": "oracle", "host": cpu,
            "sample": f"{k} full rows of A (star, n={n}, p={d}, N_ref={nref}) on {cores} single-threaded worker "
                      f"processes, {sec:.1f} s wall; each row with the kernel rows and singular-rule rows it needs; "
                      f"the regular rules of Algorithm 1 built once beforehand ({res['setup_s']:.1f} s, untimed, "
                      f"as the GPU arm builds its rules outside the timed steps)"}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on the host cores, one full row of A per
    core per step (a bounded sample of the request's assembly)."""
    if rank != 0:
        return None
    n, d, nref = args.n, args.degree, args.nref
    cpu = host_cpu()
    cores = max(1, cpu["nproc"] or 1)
    sets = [[((it * cores + q) * 7919) % n for q in range(cores)] for it in range(args.warmup + args.steps)]
    try:
        res = run_oracle(n, d, nref, sets, cores)
    except (RuntimeError, subprocess.SubprocessError) as e:
        return {"impl": "reference", "unavailable": f"oracle run failed: {str(e)[-200:]}"}
    times = res["times"][args.warmup:]
    total = sum(times)
    value = args.steps * cores * n / total
    sample = (f"{cores} full rows of A per step on {cores} single-threaded oracle worker processes "
              f"(FP64 numpy, oracle.sampled.RowSampler); rules built once, untimed ({res['setup_s']:.1f} s)")
    return {"metric": "assembled entries/s (assemble + rhs + solve per request, MIXED tier, <=1e-6 rel. error)",
            "value": value, "unit": "entries/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"star256 r=0.4(1+0.2cos5t), n={n}, p={d}, N_ref={nref}, u=log|x-(2,1)|, 1 rhs",
                       "parallelism": f"{cores} CPU processes"},
            "cpu_baseline": {"value": value, "unit": "entries/s", "cores": cores, "kind": "oracle", "host": cpu,
                             "sample": sample},
            "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    run = {"batch": run_batch, "serve": run_serve}.get(args.workload, run_ours)
    out = run(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
