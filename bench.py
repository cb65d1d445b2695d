#!/usr/bin/env python
"""Benchmark: PCG solve of the GDML force-kernel system (K + lambda I) alpha = y on GB300.

One step = the whole hot path on one synthetic system: kernel setup
(descriptors, Jacobians, distance tables, diag K), preconditioner build
(inducing-column selection + Nystrom/incomplete-Cholesky factor + Woodbury
core) and the PCG solve to TRUE relative residual 1e-8 (Sec. 2.1, Eqs. 1-5,
Alg. 1).  Default workload: N=21 atoms, M=1000 geometries (n = 63,000),
pivoted-Cholesky preconditioner with k = 2000, length scale 20, lambda 1e-10.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores instead (bounded sample, extrapolated to the full solve).
Multi-GPU (torchrun): replicas only -- every rank solves its own copy of the
system; no data-path collective exists for a single system here.
"""
from __future__ import annotations

import argparse
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

METRIC = "PCG seconds to rel. residual 1e-8 and matvec TFLOP/s, mixed vs FP64, 1 GB300"
RTOL = 1e-8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gdml", choices=["gdml", "reference"])
    ap.add_argument("--workload", default="aspirin21_m1000")
    ap.add_argument("--precision", default="ozaki", choices=["fp64", "tf32", "bf16", "df64", "ozaki"],
                    help="headline form (df64: double-float contractions on the FP32 lanes; ozaki: exact "
                         "BF16 slices on the tensor cores; both FP64-class, FP64 true-residual restarts)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the per-precision comparison solves")
    ap.add_argument("--only", default="solve", choices=["solve", "matvec", "apply", "passes", "build"],
                    help="time one operation alone (small runs for profiling); passes: the two staged "
                         "passes of the DF64/OZAKI apply on a random FP32 factor of the workload's n x k")
    ap.add_argument("--rows", type=int, default=1, choices=[1, 128, 256],
                    help="--only passes: row-chunk size of the staged passes (1: automatic)")
    ap.add_argument("--suite", default=None, choices=["batched", "learned"],
                    help="many uneven systems: per-system solves vs one batched graph solve")
    ap.add_argument("--suite-count", type=int, default=64)
    ap.add_argument("--suite-mmax", type=int, default=2000, help="cap on M (geometries) per system")
    ap.add_argument("--suite-maxiter", type=int, default=2000, help="PCG iteration cap per system in the suite")
    return ap.parse_args()


# tensor-core products per FP64-equivalent product: the sliced form multiplies
# 28 BF16 slice pairs (7 slices per operand, pairs i + j <= 8) for each one
SLICE_PAIRS = {"fp64": 1, "df64": 1, "tf32": 1, "bf16": 1, "ozaki": 28}


# ----------------------------------------------------------------- helpers
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}", "--format=csv,noheader,nounits", "-lms",
                 "200", "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------- GPU arm
def run_op(args):
    """--only matvec|apply: W untimed + K timed calls of one operation, one JSON line."""
    import torch

    from paper_2212_12737_gb300 import gdml, synth

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w = synth.workload(args.workload)
    if args.only == "passes":  # the library's test hook on a random factor (its columns contiguous)
        g = torch.Generator(device=dev).manual_seed(0)
        Lc = torch.randn(w.k, w.n, device=dev, generator=g).float()
        r = torch.randn(w.n, dtype=torch.float64, device=dev, generator=g)
        u = torch.randn(w.k, dtype=torch.float64, device=dev, generator=g)
        fn = lambda: gdml.test_df_passes(Lc.t(), r, u, w.lam, staged=args.rows)
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            fn()
        torch.cuda.synchronize(dev)
        ms = (time.perf_counter() - t0) * 1e3 / args.steps
        print(json.dumps({"op": "passes", "workload": args.workload, "rows": args.rows, "n": w.n, "k": w.k,
                          "host_ms_per_call": ms, "note": "includes the hook's scratch allocation; use ncu "
                          "kernel durations"}), flush=True)
        return
    ctx = gdml.kernel_setup(torch.from_numpy(w.R).to(dev), w.sigma, w.lam, precision=args.precision)
    if args.only == "build":  # preconditioner builds (Algorithm 1 / Nystrom + Woodbury core), host-timed
        ts = []
        for it in range(args.warmup + args.steps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            ctx.precond_build(w.select, w.k, seed=2)
            torch.cuda.synchronize(dev)
            if it >= args.warmup:
                ts.append(time.perf_counter() - t0)
        print(json.dumps({"op": "build", "workload": args.workload, "precision": args.precision,
                          "select": w.select, "k": w.k, "s": min(ts) if ts else None}), flush=True)
        ctx.destroy()
        return
    v = torch.randn(w.n, dtype=torch.float64, device=dev)
    out = torch.empty_like(v)
    if args.only == "apply":
        ctx.precond_build(w.select, w.k, seed=2)
        fn = lambda: ctx.precond_apply(v, out)
    else:
        fn = lambda: ctx.matvec(v, out)
    for _ in range(args.warmup):
        fn()
    st = torch.cuda.current_stream(dev)
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    s.record(st)
    for _ in range(args.steps):
        fn()
    e.record(st)
    torch.cuda.synchronize(dev)
    ms = s.elapsed_time(e) / args.steps
    D = w.N * (w.N - 1) // 2
    print(json.dumps({"op": args.only, "workload": args.workload, "precision": args.precision, "ms": ms,
                      "matvec_tflops": 6.0 * w.M * w.M * D / ms / 1e9 if args.only == "matvec" else None,
                      "apply_gbs": (2.0 * w.n * w.k * (4 if args.precision in ("df64", "ozaki") else 8)
                                    + 3.0 * w.k * w.k * 8) / ms / 1e6 if args.only == "apply" else None}),
          flush=True)
    ctx.destroy()


def run_suite(args):
    """Many uneven systems (N in {9,12,15,21,42}, M in [100, mmax], sigma in
    {5,10,20,40}, lambda in {1e-10,1e-8}, uniform k = M/10): per-system FP64
    solves one after another vs one batched graph solve, after autotuning."""
    import torch

    from paper_2212_12737_gb300 import gdml, synth

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    suite = synth.batched_suite(args.suite_count, mmax=args.suite_mmax)
    cache = os.path.join(ROOT, "paper_2212_12737_gb300", "lib", "tuning.json")
    ctxs, ys = [], []
    t0 = time.perf_counter()
    for w in suite:
        c = gdml.kernel_setup(torch.from_numpy(w.R).to(dev), w.sigma, w.lam)
        c.autotune(cache)
        c.precond_build("uniform", w.k, seed=2)
        ctxs.append(c)
        ys.append(torch.from_numpy(w.y).to(dev))
    torch.cuda.synchronize(dev)
    t_setup = time.perf_counter() - t0
    # warm both paths once (graph capture, instantiation)
    def seq():
        out = []
        for c, y in zip(ctxs, ys):
            _, it, rel, _ = c.pcg_solve(y, rtol=RTOL, max_iter=args.suite_maxiter, raise_on_nonconvergence=False)
            out.append((it, rel))
        return out
    t0 = time.perf_counter()
    res_seq = seq()
    torch.cuda.synchronize(dev)
    t_seq = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, its, rels = gdml.pcg_solve_batched(ctxs, ys, rtol=RTOL, max_iter=args.suite_maxiter,
                                          raise_on_nonconvergence=False)
    torch.cuda.synchronize(dev)
    t_bat = time.perf_counter() - t0
    n_tot = sum(w.n for w in suite)
    print(json.dumps({
        "suite": "batched", "systems": len(suite), "total_unknowns": n_tot, "mmax": args.suite_mmax,
        "max_iter": args.suite_maxiter,
        "setup_and_build_s": t_setup, "per_system_solves_s": t_seq, "batched_graph_solve_s": t_bat,
        "speedup": t_seq / t_bat, "iters_total": int(sum(its)),
        "converged": int(sum(r <= RTOL for r in rels)), "max_relres": max(rels),
        "same_iterations_as_per_system": all(a == b[0] for a, b in zip(its, res_seq))}), flush=True)
    for c in ctxs:
        c.destroy()


def run_learned(args):
    """Learned inducing-column scorer: train on per-geometry ridge-leverage
    labels of --suite-count training systems of the same molecule (other noise
    seeds), select k columns for the headline system, and compare PCG
    iterations / solve time with pivoted Cholesky (the fallback and referee)."""
    import torch

    from paper_2212_12737_gb300 import gdml, synth

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    base = dict(synth.WORKLOADS[args.workload])
    k = base["k"]
    t0 = time.perf_counter()
    Xs, ys = [], []
    for s in range(args.suite_count):
        cfg = dict(base)
        w = synth.make_workload(f"train{s}", cfg["N"], cfg["M"], cfg["noise"], cfg["sigma"], cfg["lam"], k,
                                "uniform", template_seed=0, noise_seed=100 + s)
        c = gdml.kernel_setup(torch.from_numpy(w.R).to(dev), w.sigma, w.lam)
        Xs.append(c.descriptors())
        ys.append(gdml.geometry_labels(c, k))
        c.destroy()
    torch.cuda.synchronize(dev)
    t_labels = time.perf_counter() - t0
    X = torch.cat(Xs)
    y = torch.cat(ys)
    sc = gdml.Scorer(X.shape[1], 256, seed=0)
    sc.fit_scaling(X, y)
    t0 = time.perf_counter()
    loss = sc.train(X, y, epochs=30, batch=256, lr=1e-3)
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t0
    w = synth.workload(args.workload)
    R = torch.from_numpy(w.R).to(dev)
    yv = torch.from_numpy(w.y).to(dev)

    def timed(fn):
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        out = fn()
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t, out

    def pivchol():
        c = gdml.kernel_setup(R, w.sigma, w.lam)
        c.precond_build("pivchol", k)
        _, it, rel, _ = c.pcg_solve(yv, rtol=RTOL, max_iter=20000, raise_on_nonconvergence=False)
        c.destroy()
        return it, rel

    def learned(referee):
        c = gdml.kernel_setup(R, w.sigma, w.lam)
        _, it, rel, used = gdml.solve_learned(c, sc, yv, k, referee_iters=referee)
        c.destroy()
        return it, rel, used

    t_pc, (it_pc, rel_pc) = timed(pivchol)
    t_l, (it_l, rel_l, used) = timed(lambda: learned(it_pc))
    # learned without the referee's cap, to report its own iteration count
    c = gdml.kernel_setup(R, w.sigma, w.lam)
    c.precond_build_scored(sc.predict(c.descriptors()), k)
    _, it_raw, rel_raw, _ = c.pcg_solve(yv, rtol=RTOL, max_iter=20000, raise_on_nonconvergence=False)
    c.destroy()
    c = gdml.kernel_setup(R, w.sigma, w.lam)
    c.precond_build("uniform", k, seed=2)
    _, it_u, rel_u, _ = c.pcg_solve(yv, rtol=RTOL, max_iter=20000, raise_on_nonconvergence=False)
    c.destroy()
    print(json.dumps({"suite": "learned", "workload": args.workload, "k": k, "train_systems": args.suite_count,
                      "label_s": t_labels, "train_s": t_train, "train_loss": loss,
                      "pivchol": {"s": t_pc, "iters": it_pc, "relres": rel_pc},
                      "learned": {"s": t_l, "iters": it_l, "relres": rel_l, "used": used,
                                  "iters_without_referee": it_raw, "relres_without_referee": rel_raw},
                      "uniform": {"iters": it_u, "relres": rel_u}}), flush=True)
    sc.destroy()


def max_over_ranks(t: float, world: int, device) -> float:
    """The job takes as long as its slowest rank: all-reduce MAX of t over the process group."""
    if world == 1:
        return t
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2212_12737_gb300 import gdml, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.workload(args.workload)
    M, N, n, k = w.M, w.N, w.n, w.k
    D = N * (N - 1) // 2
    R_h = torch.from_numpy(w.R).pin_memory()
    y_h = torch.from_numpy(w.y).pin_memory()
    R_d = R_h.to(dev)
    y_d = y_h.to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def step(prec, R, y, out_h=None):
        ctx = gdml.kernel_setup(R, w.sigma, w.lam, precision=prec)
        ctx.precond_build(w.select, k, seed=2)
        alpha, iters, rel, outer = ctx.pcg_solve(y, rtol=RTOL, max_iter=20000, raise_on_nonconvergence=False)
        if out_h is not None:
            out_h.copy_(alpha, non_blocking=True)
        ctx.destroy()
        return iters, rel, outer

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            flush.fill_(1.0)
            info = fn()
        ts = []
        barrier()
        with ClockSampler(local) as clk:
            for _ in range(steps):
                flush.fill_(2.0)  # untimed L2 flush between steps
                s = torch.cuda.Event(enable_timing=True)
                e = torch.cuda.Event(enable_timing=True)
                s.record(stream)
                info = fn()
                e.record(stream)
                torch.cuda.synchronize(dev)
                ts.append(s.elapsed_time(e) / 1e3)
        barrier()
        t = max_over_ranks(sum(ts) / len(ts), world, dev)
        return t, info, clk.summary()

    # headline: device-resident inputs
    n0 = gdml.launch_count()
    t_dev, (iters, rel, outer), clocks = timed(lambda: step(args.precision, R_d, y_d), args.steps, args.warmup)
    launches = (gdml.launch_count() - n0) // (args.steps + args.warmup)

    # e2e: host inputs, H2D + D2H inside the timed region
    alpha_h = torch.empty(n, dtype=torch.float64).pin_memory()

    def e2e_step():
        R = R_h.to(dev, non_blocking=True)
        y = y_h.to(dev, non_blocking=True)
        return step(args.precision, R, y, alpha_h)

    t_e2e, _, _ = timed(e2e_step, max(1, args.steps), 1)

    # matvec roofline: the dominant operation of every PCG iteration (6 M^2 D flop)
    def matvec_rate(prec):
        ctx = gdml.kernel_setup(R_d, w.sigma, w.lam, precision=prec)
        v = torch.randn(n, dtype=torch.float64, device=dev)
        out = torch.empty_like(v)
        for _ in range(3):
            ctx.matvec(v, out)
        reps = 20
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        s.record(stream)
        for _ in range(reps):
            ctx.matvec(v, out)
        e.record(stream)
        torch.cuda.synchronize(dev)
        ctx.destroy()
        sec = s.elapsed_time(e) / 1e3 / reps
        return sec, 6.0 * M * M * D / sec / 1e12

    def torch_peak(dtype, tf32=False, size=4096):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(size, size, device=dev, dtype=dtype)
        b = torch.randn(size, size, device=dev, dtype=dtype)
        for _ in range(2):
            a @ b
        torch.cuda.synchronize(dev)
        best = 1e9
        for _ in range(3):
            s = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record(stream)
            a @ b
            e.record(stream)
            torch.cuda.synchronize(dev)
            best = min(best, s.elapsed_time(e) / 1e3)
        torch.backends.cuda.matmul.allow_tf32 = False
        return 2.0 * size ** 3 / best / 1e12

    mv_sec, mv_tf = matvec_rate(args.precision)

    # Woodbury apply (Eq. 4): two streaming passes over L_k plus the k x k core
    def apply_rate(prec):
        ctx = gdml.kernel_setup(R_d, w.sigma, w.lam, precision=prec)
        ctx.precond_build(w.select, k, seed=2)
        v = torch.randn(n, dtype=torch.float64, device=dev)
        out = torch.empty_like(v)
        for _ in range(3):
            ctx.precond_apply(v, out)
        reps = 20
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        s.record(stream)
        for _ in range(reps):
            ctx.precond_apply(v, out)
        e.record(stream)
        torch.cuda.synchronize(dev)
        ctx.destroy()
        sec = s.elapsed_time(e) / 1e3 / reps
        lbytes = 4 if prec in ("df64", "ozaki") else 8  # FP32-stored L_k in the double-float forms
        algo = 2.0 * n * k * lbytes + 3.0 * k * k * 8
        return sec, algo

    ap_sec, ap_bytes = apply_rate(args.precision)
    peaks = measured_peaks()
    if args.precision == "fp64":
        peak, peak_src, bound = torch_peak(torch.float64), "of measured (torch FP64 matmul 4096^3, this run)", "alu"
    elif args.precision == "df64":
        # double-float on the FP32 lanes: one multiply-add (2 flop) costs ~15 FP32
        # instructions where an FP32 FMA (also 2 flop) costs one, so the ceiling is
        # the measured FP32 SIMT matmul rate / 15
        peak = torch_peak(torch.float32, tf32=False, size=8192) / 15.0
        peak_src, bound = "of derived (torch FP32 SIMT matmul 8192^3 this run / 15 FP32 ops per double-float FMA)", "alu"
    elif args.precision == "ozaki":
        # 7 BF16 slices per operand, 28 slice-pair products per contraction on tcgen05
        peak = peaks.get("bf16_tflops", 1900.0)
        peak_src, bound = "of measured (MEASURED_PEAKS.json bf16_tflops)" if peaks else "of fallback", "tensor"
    elif args.precision == "tf32":
        peak, peak_src, bound = torch_peak(torch.float32, tf32=True, size=8192), \
            "of measured (torch TF32 matmul 8192^3, this run)", "tensor"
    else:
        peak = peaks.get("bf16_tflops", 1900.0)
        peak_src, bound = "of measured (MEASURED_PEAKS.json bf16_tflops)" if peaks else "of fallback", "tensor"

    def phases(prec):
        """one solve with host-synchronised phase times (setup / build / PCG)"""
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx = gdml.kernel_setup(R_d, w.sigma, w.lam, precision=prec)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        ctx.precond_build(w.select, k, seed=2)
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
        _, it2, rel2, out2 = ctx.pcg_solve(y_d, rtol=RTOL, max_iter=20000, raise_on_nonconvergence=False)
        torch.cuda.synchronize(dev)
        t3 = time.perf_counter()
        ctx.destroy()
        return {"setup_s": t1 - t0, "build_s": t2 - t1, "solve_s": t3 - t2, "total_s": t3 - t0, "iters": it2,
                "relres": rel2, "outer": out2}

    forms = {}
    if not args.no_forms and rank == 0:
        for prec in ("fp64", "df64", "ozaki", "tf32", "bf16"):

            ph = phases(prec)
            ms2, tf2 = matvec_rate(prec)
            forms[prec] = {"s": ph["total_s"], "iters": ph["iters"], "relres": ph["relres"],
                           "converged": ph["relres"] <= RTOL, "outer": ph["outer"], "setup_s": ph["setup_s"],
                           "build_s": ph["build_s"], "solve_s": ph["solve_s"], "matvec_ms": ms2 * 1e3,
                           "matvec_tflops": tf2}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, iters)

    roof_matvec = {"kernel": f"force-kernel matvec, {args.precision} (proj + 2 contractions + back-projection)",
                   "bound": bound, "achieved": mv_tf * SLICE_PAIRS[args.precision], "peak": peak, "unit": "TFLOP/s",
                   "frac": mv_tf * SLICE_PAIRS[args.precision] / peak, "peak_source": peak_src, "traffic": None,
                   "algorithmic_flop_per_launch": 6.0 * M * M * D * SLICE_PAIRS[args.precision],
                   "fp64_equivalent_tflops": mv_tf, "matvec_ms": mv_sec * 1e3}
    hbm = peaks.get("hbm_gbs", 6800.0)
    # DRAM bytes of one apply (dram__bytes_read.sum + dram__bytes_write.sum over its 7 launches,
    # one ncu capture of `bench.py --only apply --precision ozaki` at this workload; see
    # profiles/woodbury_apply_aspirin21_m1000_k2000_ozaki.md).  Only that configuration has one.
    ap_traffic = (1040180736.0 if args.workload == "aspirin21_m1000" and args.precision in ("ozaki", "df64")
                  and w.k == 2000 else None)
    roof_apply = {"kernel": f"Woodbury apply (Eq. 4), {args.precision}: L_k^T r and L_k u passes + k x k core",
                  "bound": "hbm", "achieved": ap_bytes / ap_sec / 1e9, "peak": hbm, "unit": "GB/s",
                  "frac": ap_bytes / ap_sec / 1e9 / hbm,
                  "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "of fallback",
                  "traffic": ap_traffic, "algorithmic_bytes_per_launch": ap_bytes, "apply_ms": ap_sec * 1e3}

    if rank == 0:
        line = {
            "metric": METRIC, "value": t_dev, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_dev * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"fp64": "f64", "df64": "f32x2 (double-float) contractions + f64",
                      "ozaki": "bf16 x7 exact slices (FP32 accumulate) + f32x2 + f64", "tf32": "tf32 + f64",
                      "bf16": "bf16 + f64"}[args.precision], "data": "synthetic",
            "config": {"workload": f"{args.workload}: N={N} atoms, M={M} geometries, n={n}, D={D}, "
                                   f"{w.select} k={k}, sigma={w.sigma}, lambda={w.lam}, rtol={RTOL}",
                       "precision": args.precision, "select": w.select, "k": k, "n": n,
                       "parallelism": f"replicas x{world}",
                       "l2": "256 MB buffer written between timed steps (L2 129 MB); L_k working set "
                             f"{n * k * (4 if args.precision in ('df64', 'ozaki') else 8) / 1e9:.2f} GB"},
            "solve": {"iters": iters, "relres": rel, "outer_steps": outer, "converged": rel <= RTOL},
            "e2e": {"value": t_e2e, "unit": "s", "h2d_bytes_per_step": int(R_h.numel() * 8 + y_h.numel() * 8),
                    "d2h_bytes_per_step": int(n * 8)},
            "roofline": roof_apply if ap_sec > mv_sec else roof_matvec,
            "roofline_matvec": roof_matvec,
            "roofline_apply": roof_apply,
            "apply_ms": ap_sec * 1e3,
            "cpu_baseline": cpu,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "forms": forms,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------- CPU oracle arm
def cpu_baseline(w, gpu_iters: int, budget_s: float = 25.0):
    """Time the FP64 oracle on a bounded sample of the same solve and
    extrapolate to the full one: Alg. 1 steps (cost linear in the step index),
    matrix-free matvecs and Woodbury applies x the iteration count."""
    import numpy as np

    from oracle import kernel as ok
    from oracle import precond as op

    t0 = time.perf_counter()
    # matvec
    v = np.random.default_rng(0).standard_normal(w.n)
    reps = 0
    ts = time.perf_counter()
    while reps < 2 or (reps < 5 and time.perf_counter() - ts < 6.0):
        ok.matvec(w.R, w.sigma, v, w.lam)
        reps += 1
    t_mv = (time.perf_counter() - ts) / reps
    # Woodbury apply at the full k (cost independent of the values)
    k = w.k
    Lk = np.random.default_rng(1).standard_normal((w.n, k)) / np.sqrt(w.n)
    LC = np.linalg.cholesky(w.lam * np.eye(k) + np.eye(k))
    ts = time.perf_counter()
    op.woodbury_apply(Lk, LC, w.lam, v)
    op.woodbury_apply(Lk, LC, w.lam, v)
    t_ap = (time.perf_counter() - ts) / 2
    del Lk
    # preconditioner build sample
    if w.select == "pivchol":
        get_col = ok.column_getter(w.R, w.sigma)
        d = ok.force_kernel_diag(w.R, w.sigma)
        m1 = 40
        ts = time.perf_counter()
        op.pivoted_cholesky(get_col, d, m1)
        T1 = time.perf_counter() - ts
        ts = time.perf_counter()
        op.pivoted_cholesky(get_col, d, 2 * m1)
        T2 = time.perf_counter() - ts
        # per-step cost a + b m:  T(m) = a m + b m^2 / 2
        b = max((T2 - 2 * T1) / (m1 * m1), 0.0)
        a = max((T1 - b * m1 * m1 / 2) / m1, 0.0)
        t_build = a * k + b * k * k / 2 + 2.0 * w.n * k * k / 10e9  # + SYRK at 10 GFLOP/s
        build_note = f"Alg. 1 {m1} and {2 * m1} steps timed, fitted a+b*m per step"
    else:
        get_col = ok.column_getter(w.R, w.sigma)
        ts = time.perf_counter()
        for i in range(20):
            get_col(i)
        t_col = (time.perf_counter() - ts) / 20
        t_build = t_col * k + 3.0 * w.n * k * k / 10e9
        build_note = "20 kernel columns timed; TRSM+SYRK at 10 GFLOP/s"
    total = t_build + gpu_iters * (t_mv + t_ap)
    cores = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        cores = max(int(i.get("num_threads", 1)) for i in threadpool_info()) or cores
    except Exception:
        pass
    return {"value": total, "unit": "s", "cores": cores, "kind": "oracle",
            "sample": f"extrapolated: {reps} matrix-free matvecs ({t_mv:.3f} s), 2 Woodbury applies at k={k} "
                      f"({t_ap:.3f} s), {build_note}; x {gpu_iters} PCG iterations; sampled in "
                      f"{time.perf_counter() - t0:.1f} s"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2212_12737_gb300 import synth
    w = synth.workload(args.workload)
    # PCG iterations of the FP64 form on this system (aspirin21_m1000, pivoted Cholesky
    # k = 2000), measured by the GPU path; the oracle runs the same algorithm in FP64
    iters = int(os.environ.get("GDML_REF_ITERS", "1366"))
    vals = []
    info = None
    for i in range(args.warmup + args.steps):
        info = cpu_baseline(w, iters, budget_s=10.0)
        if i >= args.warmup:
            vals.append(info["value"])
    v = sum(vals) / len(vals)
    line = {"metric": METRIC, "value": v, "unit": "s", "impl": "reference", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "precision": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": info["cores"], "kind": "oracle",
                             "sample": info["sample"]},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.suite == "learned":
        run_learned(a)
    elif a.suite:
        run_suite(a)
    elif a.only != "solve":
        run_op(a)
    else:
        run_gpu(a)
