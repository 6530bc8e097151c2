#!/usr/bin/env python3
"""Benchmark: time to an FP64-verified relative residual of 1e-10 on the
128^3 high-contrast 7-point diffusion system (2,097,152 unknowns), AMP-PCG vs
FP64 PCG on the same kernels, one B300; HBM GB/s of the kernels.

One step = one complete solve (every row of the hot path: initial residual,
selector, scale+precondition, search direction, SpMV, updates, stopping test,
FP64 verification), inputs resident in HBM.  L2 is flushed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on the
host cores instead (bounded sample, scaled to the same metric).

--workload selects one of the further workloads instead (one JSON line each,
AMP-PCG against PCG(FP64) on the same kernels):
  elasticity96  Q1 hex elasticity, 96^3 nodes (2,626,560 dof), block CSR 3x3,
                Chebyshev degree 8, tol 1e-8
  batch512      512 independent 2D 5-point systems (sides 32..256), one
                ampcg_solve_batched call against a host loop of single solves
  adjoint64     forward + adjoint solve and dL/dtheta on the 64^3
                log-coefficient problem (L = 0.5 ||x(theta) - x_t||^2)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-10 rel. residual, AMP-PCG vs FP64 PCG on 1 B300; HBM GB/s"
TOL = 1e-10
MAXIT = 20000
GRID = 128
SIGMA = 2.0


def workload():
    import workloads as W
    a = W.diffusion3d(GRID, SIGMA, seed=0)
    b = W.rhs_uniform(a.n, seed=1)
    return a, b


def config_dict(a, extra=None):
    d = {"workload": f"{GRID}^3 7-point variable-coefficient diffusion (Dirichlet), face coeff "
                     f"exp((g_i+g_j)/2), g = 3x box-filtered N(0,1) field scaled to sigma={SIGMA}; "
                     "Jacobi; b~U[-1,1] seed 1; x0=0; tol 1e-10 FP64-verified",
         "n": int(a.n), "nnz": int(a.nnz), "coef_contrast": float(a.info["contrast"]),
         "solver": "AMP-PCG(FP16) linear criterion (ell=5, C=1), LINF_POW2 scaling, FP64 verify+replace",
         "baseline_solver": "PCG(FP64), Alg. 1, same kernels", "l2_flush": True}
    if extra:
        d.update(extra)
    return d


# DRAM bytes (read + write) per launch from one ncu capture of the kernel in
# its current form (dram__bytes_read.sum + dram__bytes_write.sum of a
# single-iteration launch on the benchmark system); a stored figure, to be
# recaptured whenever the kernel changes.  Kernels without one report null.
NCU_TRAFFIC = {"amp:iteration:uz16_ur64": 165.90e6, "amp:iteration:uz16_ur32": 97.90e6,
               "fp64:iteration:uz64_ur64": 212.40e6}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        self.f.flush()
        rows = []
        try:
            with open(self.f.name) as g:
                for line in g:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                        rows.append(parts)
        finally:
            os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def alg_bytes(kernel: str, phase: str, n: int, nnz: int, nslices: int, idx_bytes: int,
              uniform: float = 0.0) -> float:
    """Algorithmic bytes of one launch (each array the step must read or write,
    once, in the storage precision the iteration uses).  `uniform`: the
    fraction of slices stored with uniform offsets (their 8 offsets are read
    once per slice instead of an offset per entry)."""
    sz = {"64": 8, "32": 4, "16": 2}
    zb, rb = sz[phase[2:4]], sz[phase[7:9]]
    if kernel == "precond":
        # Jacobi: r, D^-1, p_{k-1} read, p_k written (z_k stays in registers)
        return n * (rb + 3 * zb)
    if kernel == "iteration":
        # k_loop: the precondition + direction, SpMV and update rows
        return sum(alg_bytes(k, phase, n, nnz, nslices, idx_bytes, uniform)
                   for k in ("precond", "spmv_gamma", "update_norm"))
    if kernel == "search_dir":
        return n * 3 * zb
    if kernel == "spmv_gamma":
        return (nnz * (rb + idx_bytes * (1.0 - uniform)) + n * (zb + rb) + nslices * 12
                + nslices * uniform * 16)
    if kernel == "update_norm":
        return n * (16 + zb + 3 * rb)
    raise KeyError(kernel)


def fp64_fmas(phase: str, n: int, nnz: int) -> float:
    """Binary64 multiply-adds of one iteration that the method itself computes
    in FP64 (Alg. 3 with the precisions of Sec. 4): with u_r = FP64 the SpMV
    (one per matrix entry), gamma, rho, the x and r updates and ||r||^2; PCG
    in FP64 adds the Jacobi product and the search direction; with u_r =
    FP32 only the x update (the inner products use Dot2 in binary32)."""
    if phase == "uz64_ur64":
        return nnz + 7.0 * n
    if phase.endswith("ur64"):
        return nnz + 5.0 * n
    return float(n)


def fp64_peak_gflops(sms: int, mhz: float) -> float:
    """FP64 pipe peak: 2 binary64 FMA per clock per SM (a single-SM probe
    measured 1.9), 2 flops per FMA, at the maximum SM clock."""
    return sms * 2 * 2 * mhz * 1e6 / 1e9


def cpu_pcg64_solve(a, b):
    """The CPU baseline: one complete solve of the benchmark system by the
    oracle's PCG (Alg. 1) in native FP64 -- the same stopping test, to an
    FP64-verified 1e-10 -- on one host core, timed end to end (no sampling,
    no extrapolation)."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.pcg64(a.rowptr, a.col, a.val, b, tol=TOL, maxit=MAXIT)
    ms = (time.perf_counter() - t0) * 1e3
    return {"kind": "oracle", "cores": 1, "value": round(ms, 1), "unit": "ms",
            "sample": f"one complete oracle FP64 PCG (Alg. 1) solve of the benchmark system, single thread: "
                      f"{r.iters} iterations, true relres {r.true_relres:.3e}",
            "iters": r.iters}


def cpu_amp_sample(a, b, iters: int = 8):
    """The oracle's AMP-PCG (software-rounded binary16/binary32, the method
    itself) timed for a bounded number of iterations on the full system; the
    per-iteration time, not a solve time."""
    import oracle
    pol = oracle.Policy(u0=oracle.FP16, criterion=oracle.LINEAR, verify_refresh=3)
    t0 = time.perf_counter()
    oracle.ampcg(a.rowptr, a.col, a.val, b, tol=TOL, maxit=1, policy=pol)
    t1 = time.perf_counter()
    oracle.ampcg(a.rowptr, a.col, a.val, b, tol=TOL, maxit=1 + iters, policy=pol)
    t2 = time.perf_counter()
    return {"per_iter_ms": round(((t2 - t1) - (t1 - t0)) / iters * 1e3, 2), "setup_ms": round((t1 - t0) * 1e3, 1),
            "iters_timed": iters, "cores": 1,
            "note": "oracle AMP-PCG(FP16) with software rounding; per-iteration time of the emulation"}


def golden_iters(key: str = "amp16_linear"):
    """Iteration count of the oracle's own solve of the benchmark system
    (tests/golden/c2_diffusion128.json, written by a script that calls only
    the oracle)."""
    p = os.path.join(ROOT, "tests", "golden", "c2_diffusion128.json")
    with open(p) as f:
        return int(json.load(f)[key]["iters"])


def max_over_ranks(vals, world: int, device: str = "cpu"):
    """Element-wise maximum of per-rank timings (the job time is the slowest
    rank's); identity on one rank."""
    if world <= 1:
        return list(vals)
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(vals), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def run_reference(args, rank, world):
    """The reference arm: the oracle (the only reference this method has; the
    paper publishes no code) on the host cores.  Each step times a bounded
    sample of oracle AMP-PCG(FP16) iterations on the full benchmark system and
    scales it to the oracle's own iteration count for the full solve (from
    the oracle-written golden file), plus the measured setup."""
    if rank != 0:
        return
    a, b = workload()
    iters = golden_iters()
    steps = []
    smp = None
    for i in range(args.warmup + args.steps):
        smp = cpu_amp_sample(a, b, iters=4)
        if i >= args.warmup:
            steps.append(smp["setup_ms"] + smp["per_iter_ms"] * iters)
    v = statistics.mean(steps)
    cb = {"kind": "oracle", "cores": 1, "value": round(v, 1), "unit": "ms",
          "sample": f"per step: 4 timed iterations of the oracle's AMP-PCG(FP16) on the full system, scaled to "
                    f"the oracle's own {iters} iterations of the full solve (tests/golden/c2_diffusion128.json)"}
    out = {"metric": METRIC, "value": round(v, 1), "unit": "ms", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(v, 1), "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f16+f32+f64 (software-rounded)", "data": "synthetic",
           "impl": "reference", "config": config_dict(a, {"iters_oracle": iters}),
           "cpu_baseline": cb,
           "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args, rank, world):
    import torch
    import paper_2505_04155_b300 as P
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    a, b = workload()
    bd = torch.as_tensor(b, device="cuda")
    s = P.Solver(a.rowptr, a.col, a.val)
    amp = P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR, verify_refresh=3)
    f64 = P.Policy.pcg64(verify_refresh=3)
    amp64w = P.Policy(u0=P.FP64, criterion=P.CRIT_WINDOW, verify_refresh=3)   # the paper's general variant
    amp_lag = P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR, verify_refresh=3, scale=P.SCALE_LINF_POW2_LAG)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    # the library's autotuner picks the iteration kernel's form per precision
    # pair on this matrix (outside the timed region)
    tuning = {"fp64_scale_none": s.tune(scale=P.SCALE_NONE, iters=20, pairs=[0]),
              "amp_scale_lag": s.tune(scale=P.SCALE_LINF_POW2_LAG, iters=20, pairs=[4, 5])}

    def timed(policy, k):
        xs, infos, ms = [], [], []
        for _ in range(k):
            flush.fill_(1.0)                      # evict L2 between steps
            x = torch.zeros_like(bd)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            x, info = s.solve(bd, x, tol=TOL, maxit=MAXIT, policy=policy, history=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            infos.append(info)
        return ms, infos, x

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # warm-up (also builds the device-side loop graph)
    timed(amp, args.warmup)
    timed(f64, args.warmup)
    timed(amp64w, args.warmup)
    timed(amp_lag, args.warmup)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        amp_ms, amp_info, x_amp = timed(amp, args.steps)
        f64_ms, f64_info, x_64 = timed(f64, args.steps)
        w_ms, w_info, _ = timed(amp64w, args.steps)
        lag_ms, lag_info, _ = timed(amp_lag, args.steps)
    barrier()
    clocks = clk.summary()
    t_amp, t_64, t_w = max_over_ranks([statistics.mean(amp_ms), statistics.mean(f64_ms), statistics.mean(w_ms)],
                                      world, "cuda")
    ia, i64 = amp_info[-1], f64_info[-1]

    # per-kernel device times (same kernels, launched one by one with events)
    _, tinfo = s.solve(bd, torch.zeros_like(bd), tol=TOL, maxit=MAXIT, policy=amp, history=False, timed=True)
    _, tinfo64 = s.solve(bd, torch.zeros_like(bd), tol=TOL, maxit=MAXIT, policy=f64, history=False, timed=True)
    peak, peak_kind = peaks()
    nslices = (a.n + 31) // 32
    lay = s.layout()
    idx_bytes = 2 if lay["idx16"] else 4
    uniform = lay["stored_uniform"] / max(lay["stored"], 1)
    kernels = {}
    for tag, ti in (("amp", tinfo), ("fp64", tinfo64)):
        ksum = sum(ti.kernel_ms.values())   # shares of kernel time, as in an ncu launch list
        for (kn, ph), ms in ti.kernel_ms.items():
            L = ti.kernel_launches_by[(kn, ph)]
            us = ms / L * 1e3
            by = alg_bytes(kn, ph, a.n, a.nnz, nslices, idx_bytes, uniform)
            kernels[f"{tag}:{kn}:{ph}"] = {"launches": L, "avg_us": round(us, 2), "alg_bytes": int(by),
                                           "gbs": round(by / (us * 1e-6) / 1e9, 1),
                                           "frac": round(by / (us * 1e-6) / 1e9 / peak, 3),
                                           "share": round(ms / ksum, 3)}
    # dominant kernel of the AMP solve
    dom = max(((k, v) for k, v in kernels.items() if k.startswith("amp:")),
              key=lambda kv: kv[1]["avg_us"] * kv[1]["launches"])
    dk, dv = dom
    achieved = dv["gbs"]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 3), "traffic": NCU_TRAFFIC.get(dk),
                "traffic_source": "stored ncu dram bytes (read + write) of one launch of this kernel", "kernel": dk,
                "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}

    # per-iteration device time inside the loop graph, per precision pair:
    # fixed-pair solves of FIXED_ITERS iterations (tolerance out of reach), L2
    # flushed before each, CUDA events around the solve
    FIXED_ITERS = 400
    graph_iter = {}
    lagp = dict(scale=P.SCALE_LINF_POW2_LAG)
    for ph, pol in (("uz16_ur64", P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=P.FP64)),
                    ("uz16_ur32", P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=P.FP32)),
                    ("uz16_ur64_lag", P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=P.FP64, **lagp)),
                    ("uz16_ur32_lag", P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=P.FP32, **lagp)),
                    ("uz64_ur64", P.Policy.pcg64())):
        best = None
        for _ in range(3):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            _, fi = s.solve(bd, torch.zeros_like(bd), tol=1e-300, maxit=FIXED_ITERS, policy=pol, history=False)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) * 1e3 / max(fi.iters, 1)
            best = t if best is None else min(best, t)
        by = alg_bytes("iteration", ph[:9], a.n, a.nnz, nslices, idx_bytes, uniform)
        graph_iter[ph] = {"us": round(best, 2), "alg_bytes": int(by), "gbs": round(by / (best * 1e-6) / 1e9, 1),
                          "frac": round(by / (best * 1e-6) / 1e9 / peak, 3)}

    # the same dominant kernel against the FP64 pipe: the Phase-1 iteration
    # (and PCG's) carries the method's binary64 multiply-adds, and ncu shows
    # that pipe, not DRAM, as its busiest unit
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = 2032.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except (OSError, ValueError):
        pass
    fpk = fp64_peak_gflops(sms, mhz)
    dph = dk.split(":")[2]
    fl = 2.0 * fp64_fmas(dph, a.n, a.nnz)
    roofline_fp64 = {"bound": "alu", "pipe": "fp64", "kernel": dk,
                     "achieved": round(fl / (dv["avg_us"] * 1e-6) / 1e9, 1), "peak": round(fpk, 1),
                     "unit": "GFLOP/s", "frac": round(fl / (dv["avg_us"] * 1e-6) / 1e9 / fpk, 3),
                     "flops_per_launch": int(fl),
                     "in_graph": {k: {"gflops": round(2.0 * fp64_fmas(k[:9], a.n, a.nnz) / (v["us"] * 1e-6) / 1e9, 1),
                                      "frac": round(2.0 * fp64_fmas(k[:9], a.n, a.nnz) / (v["us"] * 1e-6) / 1e9 / fpk,
                                                    3)}
                                  for k, v in graph_iter.items()},
                     "peak_kind": f"derived: {sms} SMs x 2 FP64 FMA per clock x 2 flops x {mhz:.0f} MHz"}
    # the bench line's roofline is the binding one: the roof with the longer
    # floor time for the dominant kernel's algorithmic work (the Phase-1
    # iteration sits at the FP64 ridge point, 0.2 flop per byte, with the FP64
    # floor slightly above the HBM floor; ncu: FP64 pipe 60% busy, DRAM 24%)
    roofline_hbm = roofline
    t_hbm = dv["alg_bytes"] / (peak * 1e9)
    t_fp64 = fl / (fpk * 1e9)
    if t_fp64 > t_hbm:
        roofline = {"bound": "alu", "pipe": "fp64", "achieved": round(roofline_fp64["achieved"] / 1e3, 4),
                    "peak": round(fpk / 1e3, 4), "unit": "TFLOP/s", "frac": roofline_fp64["frac"],
                    "traffic": NCU_TRAFFIC.get(dk), "traffic_source": roofline_hbm["traffic_source"], "kernel": dk,
                    "peak_kind": roofline_fp64["peak_kind"],
                    "floor_us": {"fp64": round(t_fp64 * 1e6, 2), "hbm": round(t_hbm * 1e6, 2)}}

    # the choice of omega_k (Sec. 3.3; reading R5): the same AMP-PCG(FP16)
    # solve under omega = 1/||r_k|| (Alg. 3 as printed), the exact power of two
    # 2^-ceil(log2 max|r_k|) (the default) and the lagged one (reading R20),
    # GPU time and iterations beside the oracle's iterations and binary16
    # underflow fractions (an oracle-written file)
    study = {}
    oracle_study = {}
    sp = os.path.join(ROOT, "tests", "golden", "c2_scale_study.json")
    if os.path.exists(sp):
        with open(sp) as f:
            oracle_study = json.load(f)
    for name, sc in (("L2", P.SCALE_L2), ("LINF_POW2", P.SCALE_LINF_POW2), ("LINF_POW2_LAG", P.SCALE_LINF_POW2_LAG)):
        pol = P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR, verify_refresh=3, scale=sc)
        timed(pol, 1)
        ms_, inf_, _ = timed(pol, 3)
        o = oracle_study.get(name, {})
        study[name] = {"ms": round(statistics.mean(ms_), 3), "iters": inf_[-1].iters,
                       "switch_iter": list(inf_[-1].switch_iter), "true_relres": inf_[-1].true_relres,
                       "oracle_iters": o.get("iters"),
                       "oracle_y16_below_normal_frac": o.get("y16_below_normal_frac")}

    # end to end through the C ABI with pinned host buffers
    bh = torch.as_tensor(b).pin_memory()
    xh = torch.zeros(a.n, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.fill_(1.0)
        xh.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, einfo = s.solve(bh, xh, tol=TOL, maxit=MAXIT, policy=amp, history=False)
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e = {"value": statistics.mean(e2e_ms), "unit": "ms", "h2d_bytes_per_step": int(16 * a.n),
           "d2h_bytes_per_step": int(8 * a.n), "note": "wall clock around ampcg_solve with pinned host b, x"}

    out = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu:
            cpu = cpu_pcg64_solve(a, b)
            cpu["amp_emulation"] = cpu_amp_sample(a, b)
        launches = int(sum(i.kernel_launches for i in amp_info + f64_info + w_info + lag_info))
        out = {"metric": METRIC, "value": round(t_amp, 3), "unit": "ms", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_amp, 3),
               "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
               "dtype": "f16+f32+f64", "data": "synthetic",
               "config": config_dict(a, {"parallelism": "replicas" if world > 1 else "single"}),
               "fp64_pcg_ms": round(t_64, 3), "speedup_vs_fp64_pcg": round(t_64 / t_amp, 3),
               "iters_amp": ia.iters, "iters_fp64": i64.iters, "refreshes_amp": ia.refreshes,
               "true_relres_amp": ia.true_relres, "true_relres_fp64": i64.true_relres,
               "switch_iter_amp": list(ia.switch_iter),
               "amp_lag_ms": round(statistics.mean(lag_ms), 3), "iters_amp_lag": lag_info[-1].iters,
               "switch_iter_amp_lag": list(lag_info[-1].switch_iter), "true_relres_amp_lag": lag_info[-1].true_relres,
               "amp64_window_ms": round(t_w, 3), "iters_amp64_window": w_info[-1].iters,
               "switch_iter_amp64_window": list(w_info[-1].switch_iter),
               "true_relres_amp64_window": w_info[-1].true_relres,
               "roofline": roofline, "roofline_hbm": roofline_hbm, "roofline_fp64": roofline_fp64, "kernels": kernels, "cpu_baseline": cpu,
               "e2e": e2e,
               "clocks": clocks, "gpu_launches": launches,
               "iteration_in_graph": graph_iter, "layout": lay, "autotune": tuning, "scale_study": study,
               "gpu_launches_note": "library kernels in the timed region (all timed solves), counted by the library"}
        print(json.dumps(out), flush=True)
    s.close()
    return out


def _event_ms(fn, k, flush):
    """Mean device time of k calls of fn (L2 flushed before each)."""
    import torch
    stream = torch.cuda.current_stream()
    ms, out = [], None
    for _ in range(k):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.mean(ms), out


def run_workload(args):
    """The further workloads (--workload); rank 0, one GPU."""
    import torch
    import paper_2505_04155_b300 as P
    import workloads as W
    torch.cuda.set_device(0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    amp = P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR, verify_refresh=3)
    f64 = P.Policy.pcg64(verify_refresh=3)
    base = {"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16+f32+f64", "data": "synthetic"}
    if args.workload == "elasticity96":
        t0 = time.time()
        a = W.elasticity_q1(96, seed=0)
        b = W.rhs_uniform(a.nb * 3, seed=1)
        gen_s = time.time() - t0
        s = P.Solver.from_bsr(a.browptr, a.bcol, a.bval, 3, precond=P.M_CHEBYSHEV, degree=8)
        bd = torch.as_tensor(b, device="cuda")
        run = lambda pol: s.solve(bd, torch.zeros_like(bd), tol=1e-8, maxit=MAXIT, policy=pol, history=False)
        for _ in range(args.warmup):
            run(amp), run(f64)
        ta, (_, ia) = _event_ms(lambda: run(amp), args.steps, flush)
        t6, (_, i6) = _event_ms(lambda: run(f64), args.steps, flush)
        lmin, lmax = s.interval()
        s.close()
        out = {"metric": "time-to-1e-8 rel. residual, Q1 elasticity (block CSR 3x3, Chebyshev degree 8), "
                         "AMP-PCG vs FP64 PCG on 1 B300",
               "value": round(ta, 3), "unit": "ms", "ms_per_step": round(ta, 3),
               "config": {"workload": "Q1 hex elasticity 96^3 nodes, x=0 face clamped, E log-uniform "
                                      "[1,1e3] per element (seed 0), nu=0.3; b~U[-1,1] seed 1; x0=0",
                          "dof": int(a.nb * 3), "nnzb": int(len(a.bcol)), "cheb_interval": [lmin, lmax],
                          "generator_s": round(gen_s, 1), "l2_flush": True},
               "fp64_pcg_ms": round(t6, 3), "speedup_vs_fp64_pcg": round(t6 / ta, 3),
               "iters_amp": ia.iters, "iters_fp64": i6.iters, "switch_iter_amp": list(ia.switch_iter),
               "true_relres_amp": ia.true_relres, "true_relres_fp64": i6.true_relres,
               "refreshes_amp": ia.refreshes}
    elif args.workload == "batch512":
        mats, rhs = W.batch_2d(512, seed=0)
        ss = [P.Solver(m.rowptr, m.col, m.val) for m in mats]
        bs = [torch.as_tensor(r, device="cuda") for r in rhs]
        xs = [torch.zeros_like(b) for b in bs]

        def batched(pol):
            for x in xs:
                x.zero_()
            return P.solve_batched(ss, bs, xs, tol=1e-10, maxit=MAXIT, policy=pol)

        # the library's autotuner picks the batched kernel's block size (outside the timed region)
        btune = P.tune_batched(ss, iters=40, policy=amp)

        def loop(pol):
            return [s.solve(b, torch.zeros_like(b), tol=1e-10, maxit=MAXIT, policy=pol, history=False)[1]
                    for s, b in zip(ss, bs)]

        for _ in range(args.warmup):
            batched(amp), loop(amp), batched(f64)
        tb, ib = _event_ms(lambda: batched(amp), args.steps, flush)
        tl, il = _event_ms(lambda: loop(amp), args.steps, flush)
        tb6, ib6 = _event_ms(lambda: batched(f64), args.steps, flush)
        amp_lag = P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR, verify_refresh=3, scale=P.SCALE_LINF_POW2_LAG)
        batched(amp_lag)
        tbl, ibl = _event_ms(lambda: batched(amp_lag), args.steps, flush)
        same = all(i.iters == j.iters for i, j in zip(ib, il))
        for s in ss:
            s.close()
        n_tot = int(sum(m.n for m in mats))
        out = {"metric": "time to solve 512 independent 2D systems to 1e-10 (FP64-verified), "
                         "one batched call vs a host loop of single solves, 1 B300",
               "value": round(tb, 3), "unit": "ms", "ms_per_step": round(tb, 3),
               "config": {"workload": "512 systems, 2D 5-point, side ~ U{32..256} (seed 0), cell coeffs "
                                      "exp(N(0,1)) (seed 1000+i), faces geometric mean; b_i~U[-1,1]",
                          "sum_n": n_tot, "sum_nnz": int(sum(m.nnz for m in mats)),
                          "solver": "AMP-PCG(FP16) linear criterion, Jacobi", "l2_flush": True},
               "host_loop_ms": round(tl, 3), "speedup_vs_host_loop": round(tl / tb, 3),
               "fp64_batched_ms": round(tb6, 3), "speedup_vs_fp64_batched": round(tb6 / tb, 3),
               "amp_lag_batched_ms": round(tbl, 3), "iters_max_amp_lag": max(i.iters for i in ibl),
               "all_converged_amp_lag": all(i.converged for i in ibl),
               "iters_max": max(i.iters for i in ib), "iters_mean": round(statistics.mean(i.iters for i in ib), 1),
               "all_converged": all(i.converged for i in ib), "batched_iters_equal_single": same,
               "unknowns_per_s": round(n_tot / (tb * 1e-3), 1), "autotune": btune}
    else:  # adjoint64
        from paper_2505_04155_b300 import autograd as AG
        theta, theta_t, a, a_t, b = W.log_coeff_problem(64, sigma=1.0, seed=0)
        s = P.Solver(a.rowptr, a.col, a.val)
        st = P.Solver(a_t.rowptr, a_t.col, a_t.val)
        nb = torch.as_tensor(a.info["nbound"], device="cuda")
        bd = torch.as_tensor(b, device="cuda")
        x_t, _ = st.solve(bd, tol=1e-13, maxit=MAXIT, policy=P.Policy.pcg64())
        st.close()
        th0 = torch.as_tensor(theta, device="cuda")

        def grad(pol):
            th = th0.clone().requires_grad_(True)
            x = AG.solve_log_coeff(th, bd, s, nb, tol=1e-10, maxit=MAXIT, policy=pol)
            L = 0.5 * torch.sum((x - x_t) ** 2)
            L.backward()
            return th.grad

        for _ in range(args.warmup):
            grad(amp), grad(f64)
        ta, ga = _event_ms(lambda: grad(amp), args.steps, flush)
        amp_lag = P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR, verify_refresh=3, scale=P.SCALE_LINF_POW2_LAG)
        s.tune(scale=P.SCALE_LINF_POW2_LAG, iters=20, pairs=[4, 5])
        s.tune(scale=P.SCALE_NONE, iters=20, pairs=[0])
        grad(amp_lag)
        tl, gl = _event_ms(lambda: grad(amp_lag), args.steps, flush)
        t6, g6 = _event_ms(lambda: grad(f64), args.steps, flush)
        rel = float(torch.linalg.norm(ga - g6) / torch.linalg.norm(g6))
        s.close()
        out = {"metric": "time of one dL/dtheta evaluation (forward solve + adjoint solve + gradient "
                         "assembly) to 1e-10, AMP-PCG vs FP64 PCG on 1 B300",
               "value": round(ta, 3), "unit": "ms", "ms_per_step": round(ta, 3),
               "config": {"workload": "64^3 7-point log-coefficient diffusion, theta = 3x box-filtered "
                                      "N(0,1) field, sigma=1 (seed 0); theta_t = theta + 0.1 field (seed 2); "
                                      "b~U[-1,1] seed 1; L = 0.5||x(theta) - x_t||^2",
                          "n": int(a.n), "nnz": int(a.nnz), "l2_flush": True},
               "fp64_ms": round(t6, 3), "speedup_vs_fp64": round(t6 / ta, 3),
               "grad_rel_diff_amp_vs_fp64": rel, "amp_lag_ms": round(tl, 3),
               "grad_rel_diff_amp_lag_vs_fp64": float(torch.linalg.norm(gl - g6) / torch.linalg.norm(g6))}
    out.update(base)
    print(json.dumps(out), flush=True)


def run_profile(args):
    """One solve of the benchmark system for a profiler, with the iteration
    kernels launched one by one (ampcg_solve_timed: the same kernels and
    iterates as the graph path; profilers cannot see kernel nodes of graphs
    with conditional nodes).  `amp` is the benchmarked AMP-PCG policy;
    `p1`/`p2`/`fp64` pin the precision pair of Phase 1 (u_z=FP16, u_r=FP64),
    Phase 2 (FP16, FP32) or PCG(FP64): the AMP pairs under the benchmark's
    exact power-of-two scale in the three-barrier iteration kernel the
    benchmark runs, PCG(FP64) in the four-barrier one its tuner keeps;
    `p1_four`/`p2_four` the AMP pairs in the four-barrier kernel;
    `p1_lag`/`p2_lag` the same pairs under the lagged scale."""
    import torch
    import paper_2505_04155_b300 as P
    torch.cuda.set_device(0)
    if args.profile.startswith("batch"):
        # persistent batched kernel: 16 systems of 256 x 256 (the batch's largest
        # size), Phase 1 or Phase 2 precisions, profile_iters iterations
        import workloads as W
        mats = [W.diffusion2d_cells(256, 1000 + i) for i in range(16)]
        ss = [P.Solver(m.rowptr, m.col, m.val) for m in mats]
        bs = [torch.as_tensor(W.rhs_uniform(m.n, i), device="cuda") for i, m in enumerate(mats)]
        xs = [torch.zeros_like(v) for v in bs]
        ur = P.FP64 if args.profile == "batch_p1" else P.FP32
        pol = P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=ur)
        t0 = time.perf_counter()
        infos = P.solve_batched(ss, bs, xs, tol=TOL, maxit=args.profile_iters or 40, policy=pol)
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "iters": infos[0].iters,
                          "ms": round((time.perf_counter() - t0) * 1e3, 3)}), flush=True)
        for s in ss:
            s.close()
        return
    if args.profile.startswith("cheb"):
        # Chebyshev(8) on block-CSR Q1 elasticity, 48^3 nodes (330K dof), Phase 2 or
        # FP64 precisions, profile_iters iterations, kernels launched one by one
        import workloads as W
        e = W.elasticity_q1(48, seed=0)
        s = P.Solver.from_bsr(e.browptr, e.bcol, e.bval, 3, precond=P.M_CHEBYSHEV, degree=8)
        bd = torch.as_tensor(W.rhs_uniform(e.nb * 3, seed=1), device="cuda")
        pol = (P.Policy.pcg64() if args.profile == "cheb_fp64"
               else P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=P.FP32))
        _, info = s.solve(bd, tol=1e-8, maxit=args.profile_iters or 20, policy=pol, history=False, timed=True)
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "iters": info.iters,
                          "kernel_us": {f"{k[0]}:{k[1]}": round(v / info.kernel_launches_by[k] * 1e3, 2)
                                        for k, v in info.kernel_ms.items()}}), flush=True)
        s.close()
        return
    a, b = workload()
    s = P.Solver(a.rowptr, a.col, a.val)
    lag = P.SCALE_LINF_POW2_LAG
    pol = {"amp": P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR, verify_refresh=3),
           "p1": P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=P.FP64),
           "p2": P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=P.FP32),
           "p1_four": P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=P.FP64),
           "p2_four": P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=P.FP32),
           "p1_lag": P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=P.FP64, scale=lag),
           "p2_lag": P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=P.FP32, scale=lag),
           "fp64": P.Policy.pcg64()}[args.profile]
    if args.profile == "fp64":
        s.set_tuning([0] * 6, scale=P.SCALE_NONE)   # the form the autotuner keeps for FP64 PCG
    if args.profile.endswith("_four"):
        s.set_tuning([0] * 6, scale=P.SCALE_LINF_POW2)
    maxit = args.profile_iters if args.profile_iters > 0 else MAXIT
    bd = torch.as_tensor(b, device="cuda")
    _, info = s.solve(bd, tol=TOL, maxit=maxit, policy=pol, history=False, timed=True)
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "iters": info.iters, "status": info.status,
                      "true_relres": info.true_relres, "launches": info.kernel_launches,
                      "kernel_us": {f"{k[0]}:{k[1]}": round(v / info.kernel_launches_by[k] * 1e3, 2)
                                    for k, v in info.kernel_ms.items()}}), flush=True)
    s.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--profile", choices=["amp", "p1", "p2", "p1_four", "p2_four", "p1_lag", "p2_lag", "fp64",
                                          "batch_p1", "batch_p2", "cheb_p2", "cheb_fp64"],
                    default=None,
                    help="run one solve for a profiler and exit")
    ap.add_argument("--profile-iters", type=int, default=0, help="maxit of the profiled solve (0: converge)")
    ap.add_argument("--workload", choices=["diffusion128", "elasticity96", "batch512", "adjoint64"],
                    default="diffusion128", help="diffusion128: the headline benchmark")
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
        return
    if args.workload != "diffusion128":
        if int(os.environ.get("RANK", "0")) == 0:
            run_workload(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
