#!/usr/bin/env python3
"""Benchmark: matrix-free CP-ALS of the DF particle-particle-ladder tensor on GB300.

Workload: one PPL instance with o=20 occupied, v=200 virtual, X=600 auxiliary
orbitals and CP rank R=800, seeded synthetic inputs shaped like the paper's
molecules (paper_2503_10380_gb300/inputs.py).  One step = one ALS sweep
(modes a, b, i, j) with TF32x3 tensor-core MTTKRPs (tf32 hi/lo split,
accumulator restarted every K block) and FP64 Gram / Cholesky / solve / fit.
BF16x3 is timed beside it with its energy error.  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload single|batch|precision|sequence] [--precision bf16x3|tf32|tf32x3]

For N > 1 (one process per GPU under torchrun) every rank runs an
independent replica (the method has no exchange step on one instance):
value = N * K / max over ranks of the timed region.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CP-ALS sweeps/s & MTTKRP TFLOP/s at ≤0.1 kcal/mol ΔE vs plain FP64 on GPU"
O, V, XAUX, RANK, SEED = 20, 200, 600, 800, 0
SWEEPS_PER_SOLVE = 30          # the configuration's ALS sweep count
KCAL = 627.509474
WORKLOAD = f"cp-als-ppl single instance o={O} v={V} X={XAUX} R={RANK}, {SWEEPS_PER_SOLVE} sweeps per solve"


def alg_flops(o, v, X, R):
    """Algorithmic MTTKRP flops of one sweep: 4 o^2 v^2 R + 16 X v^2 R."""
    return 4.0 * o * o * v * v * R + 16.0 * X * v * v * R


def reduce_max(x: float, world: int, dev=None) -> float:
    """Max over ranks (the slowest replica sets the whole-job time)."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev if dev is not None else "cpu")
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def oracle_cores():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n)), "threadpoolctl"
    except Exception:
        pass
    return os.cpu_count() or 1, "nproc (BLAS default thread count)"


def time_oracle_sweeps(inp, R_s, nsweeps):
    """Time `nsweeps` FP64 oracle sweeps of the rank-R_s problem on the host cores."""
    import numpy as np
    from oracle import ppl_oracle as orc
    U = {m: inp.factors[m][:, :R_s].copy() for m in orc.MODES}
    lam = np.ones(R_s)
    Bvv = np.ascontiguousarray(inp.Bvv)
    t0 = time.perf_counter()
    for _ in range(nsweeps):
        U, lam, _ = orc.als_sweep(Bvv, inp.tau, U, lam)
    return time.perf_counter() - t0


def oracle_estimate(o, v, X, R):
    """CPU baseline for a size too large to time the oracle on: one FP64 oracle sweep of
    the o=20 v=200 X=600 R=800 instance is timed on the host cores and its MTTKRP-flop
    rate is scaled to (o, v, X, R).  Labelled as an estimate."""
    from paper_2503_10380_gb300 import inputs
    inp = inputs.make_inputs(O, V, XAUX, RANK, seed=SEED)
    t = time_oracle_sweeps(inp, RANK, 1)
    rate = alg_flops(O, V, XAUX, RANK) / t
    cores, how = oracle_cores()
    return {"value": rate / alg_flops(o, v, X, R), "unit": "sweeps/s", "cores": cores, "kind": "oracle",
            "estimate": True,
            "sample": f"estimate: one FP64 oracle sweep of o={O} v={V} X={XAUX} R={RANK} took {t:.2f} s "
                      f"({rate / 1e9:.1f} GFLOP/s of MTTKRP flops), scaled by 4o^2v^2R + 16Xv^2R to "
                      f"o={o} v={v} X={X} R={R}; threads from {how}"}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                if int(f[0]) != self.idx:
                    continue
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def traffic_from_profile(key: str, src_name: str):
    """DRAM bytes from the committed ncu summary (profiles/mttkrp_tc_cfg1_traffic.json)
    if it was taken on the current source of the kernel; else None."""
    src = os.path.join(ROOT, "paper_2503_10380_gb300", "csrc", src_name)
    prof = os.path.join(ROOT, "profiles", "mttkrp_tc_cfg1_traffic.json")
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        d = json.load(open(prof))
        if d.get(src_name.replace(".cu", "") + "_sha256") == h:
            return d.get(key)
    except Exception:
        pass
    return None


def tensor_peak(pk, precision):
    """Algorithmic-flop peak of a tensor-core precision: the dtype's sustained
    rate divided by the MMAs issued per product (three for the split forms)."""
    bf16 = pk["bf16_tflops_sustained"]
    tf32 = bf16 * (1.1 / 2.25)          # nominal dense tf32 / bf16 ratio
    return {"bf16x3": (bf16 / 3.0, "sustained bf16 / 3 (three bf16 MMAs per product)"),
            "tf32": (tf32, "sustained bf16 x nominal tf32/bf16 ratio 1.1/2.25"),
            "tf32x3": (tf32 / 3.0, "sustained bf16 x nominal tf32/bf16 ratio 1.1/2.25, / 3 (three tf32 MMAs "
                                   "per product)")}[precision]


def fp64_solve_flops(o, v, R):
    """Algorithmic FP64 flops of the four mode updates of one sweep: per mode
    2 R^3 / 3 (Cholesky) + 3 dim R^2 (forward and back substitution, Gram)."""
    return 4 * (2.0 * R ** 3 / 3.0) + 3.0 * R * R * (2 * v + 2 * o)


def fp64_peak_tflops(pk):
    """FP64 FMA peak derived from ncu's sm__sass_thread_inst_executed_op_dfma_pred_on
    peak_sustained = 2 per clock per SM: 2 FMA x 2 flops x SMs x max SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return 2 * 2 * sms * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def run_reference(args, world, rank):
    if rank != 0:
        return
    from paper_2503_10380_gb300 import inputs
    inp = inputs.make_inputs(O, V, XAUX, RANK, seed=SEED)
    # size each step to the budget: a step is one oracle sweep over the first
    # R_s rank columns (all of them when the budget allows); per-r work is
    # independent, so sweeps/s of the full problem = (R_s / R) / step time
    budget = 150.0
    t_cal = time_oracle_sweeps(inp, 64, 1)
    per_col = t_cal / 64
    R_s = int(max(16, min(RANK, (budget / max(args.steps + args.warmup, 1)) / per_col)))
    for _ in range(args.warmup):
        time_oracle_sweeps(inp, R_s, 1)
    t = time_oracle_sweeps(inp, R_s, args.steps)
    value = (args.steps * R_s / RANK) / t
    cores, how = oracle_cores()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded; shapes of the paper's molecules)",
        "config": {"workload": WORKLOAD, "o": O, "v": V, "X": XAUX, "R": RANK},
        "cpu_baseline": {"value": value, "unit": "sweeps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} FP64 oracle sweeps over the first {R_s} of {RANK} rank columns, "
                                   f"scaled by {R_s}/{RANK}; threads from {how}"},
        "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    from paper_2503_10380_gb300 import binding, inputs
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    binding.lib()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    inp = inputs.make_inputs(O, V, XAUX, RANK, seed=SEED)
    B_h = torch.from_numpy(inp.B).pin_memory()
    tau_h = torch.from_numpy(inp.tau).pin_memory()
    B = B_h.to(dev)
    tau = tau_h.to(dev)
    stream = torch.cuda.current_stream(dev)

    cp = binding.CpAls(B, tau, inp.factors, precision=args.precision, profile=True, r_chunk=args.r_chunk)
    if not args.r_chunk:
        args.r_chunk = cp.autotune()       # the library's own r-chunk autotuner (before the timed region)
    normR2, E_exact, _ = cp.exact_contract()
    for _ in range(args.warmup):
        cp.sweep(1, want_hist=False)
    torch.cuda.synchronize()

    # ---- timed region: K back-to-back graph-replayed sweeps -------------------
    clocks = ClockSampler(local)
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    cp.sweep(args.steps, want_hist=False)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    ms = reduce_max(e0.elapsed_time(e1), world, dev)
    ms_per_step = ms / args.steps
    value = world * args.steps / (ms / 1000.0)
    st = cp.stats()
    fit_last = st["last_fit"]

    # ---- phase breakdown (CUDA events recorded by the library on its stream) --
    nprof = min(args.steps, 5)
    acc = None
    for _ in range(nprof):
        cp.sweep(1, want_hist=False)
        ph = cp.phase_ms()
        acc = ph if acc is None else {k: acc[k] + ph[k] for k in acc}
    phases = {k: acc[k] / nprof for k in acc}
    mttkrp_ms = phases["tau_r"] + phases["chain_a"] + phases["chain_b"] + phases["s_and_p"]
    flops = alg_flops(O, V, XAUX, RANK)
    mttkrp_tflops = flops / (mttkrp_ms / 1000.0) / 1e12
    cp.close()

    # ---- accuracy and the plain FP64 GPU form from the same start -------------
    n_cmp = SWEEPS_PER_SOLVE
    mixed = binding.CpAls(B, tau, inp.factors, precision=args.precision, r_chunk=args.r_chunk)
    mixed.set_normR2(normR2)
    M_mixed = mixed.mttkrp("a")              # one MTTKRP from the initial guess, before any sweep
    fits_mixed = mixed.sweep(n_cmp)
    E_mixed = mixed.energy()
    mixed.close()
    f64 = binding.CpAls(B, tau, inp.factors, precision="fp64")
    f64.set_normR2(normR2)
    M_f64 = f64.mttkrp("a")

    def mttkrp_err(M):
        return float(torch.linalg.norm(M - M_f64) / torch.linalg.norm(M_f64))
    f64.sweep(1, want_hist=False)          # capture
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    fits_f64 = f64.sweep(n_cmp - 1)
    g1.record(stream)
    torch.cuda.synchronize()
    f64_ms = g0.elapsed_time(g1) / (n_cmp - 1)
    E_f64 = f64.energy()
    f64.close()

    # ---- the other tensor-core precisions on the same start: speed and accuracy
    variants = {}
    for prec in ("bf16x3", "tf32x3"):
        if prec == args.precision:
            continue
        alt = binding.CpAls(B, tau, inp.factors, precision=prec, r_chunk=args.r_chunk)
        alt.set_normR2(normR2)
        alt_err = mttkrp_err(alt.mttkrp("a"))
        alt.sweep(n_cmp, want_hist=False)
        E_alt = alt.energy()
        torch.cuda.synchronize()
        g0.record(stream)
        alt.sweep(50, want_hist=False)
        g1.record(stream)
        torch.cuda.synchronize()
        variants[prec] = {"sweeps_per_s": 50 * 1000.0 / g0.elapsed_time(g1), "E_cp": E_alt,
                          "mttkrp_rel_err": alt_err,
                          "dE_kcal_per_mol": abs(E_alt - E_f64) * KCAL,
                          "meets_0.1_kcal": abs(E_alt - E_f64) * KCAL <= 0.1}
        alt.close()

    # ---- end to end through the C ABI with host buffers -----------------------
    # per solve (one CC-like iteration): tau copied from pinned host memory,
    # its operand copies rebuilt, SWEEPS_PER_SOLVE sweeps warm-started from the
    # factors already on the device, then factors and fit history read back.
    # B stays resident (the DF integrals do not change between CC iterations).
    e2e = binding.CpAls(B, tau, inp.factors, precision=args.precision, r_chunk=args.r_chunk)
    e2e.set_normR2(normR2)
    fac_out = torch.empty(e2e.fac.numel(), dtype=torch.float64).pin_memory()
    tau_dev = e2e.tau

    def e2e_step():
        tau_dev.copy_(tau_h, non_blocking=True)
        binding.ppl_cpd_set_tau(e2e.h, tau_dev.data_ptr())
        hist = e2e.sweep(SWEEPS_PER_SOLVE, want_hist=True)
        fac_out.copy_(e2e.fac, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
        return hist

    e2e_step()
    n_e2e = 3
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_step()
    torch.cuda.synchronize()
    t_e2e = reduce_max(time.perf_counter() - t0, world, dev)
    e2e.close()
    e2e_value = world * n_e2e * SWEEPS_PER_SOLVE / t_e2e
    h2d = tau_h.numel() * 8
    d2h = fac_out.numel() * 8 + SWEEPS_PER_SOLVE * 8

    # ---- CPU baseline: the oracle on the host cores (rank 0, N = 1) -----------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_or = 2
        t_or = time_oracle_sweeps(inp, RANK, n_or)
        cores, how = oracle_cores()
        cpu = {"value": n_or / t_or, "unit": "sweeps/s", "cores": cores, "kind": "oracle",
               "sample": f"{n_or} full FP64 oracle sweeps of the same o={O} v={V} X={XAUX} R={RANK} instance; "
                         f"threads from {how}"}

    pk, pk_kind = peaks()
    peak, peak_note = tensor_peak(pk, args.precision)
    # DRAM bytes per sweep of each roofline's kernels (the same per-sweep unit as `achieved`)
    traffic_mttkrp = traffic_from_profile("mttkrp_bytes_per_sweep", "ppl_tc.cu")
    traffic_solve = traffic_from_profile("solve_bytes_per_sweep", "ppl_solve.cu")
    solve_ms = phases["solve_a"] + phases["solve_b"] + phases["solve_ij"]
    solve_tflops = fp64_solve_flops(O, V, RANK) / (solve_ms / 1000.0) / 1e12
    fp64_peak = fp64_peak_tflops(pk)
    roof_solve = {"bound": "alu", "achieved": solve_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                  "frac": solve_tflops / fp64_peak, "traffic": traffic_solve, "ms_per_sweep": solve_ms,
                  "kernel": "k_solve (FP64 mode updates, cooperative, 4 launches per sweep)",
                  "peak_source": "derived: 2 DFMA/clk/SM (ncu peak_sustained) x 2 flops x SMs x max SM clock",
                  "work": "per sweep 4 x 2R^3/3 + 3 R^2 (2v + 2o) FP64 flops"}
    roof_mttkrp = {"bound": "tensor", "achieved": mttkrp_tflops, "peak": peak, "unit": "TFLOP/s",
                   "frac": mttkrp_tflops / peak, "traffic": traffic_mttkrp, "ms_per_sweep": mttkrp_ms,
                   "kernel": "k_tc_gemm and its helpers (all MTTKRP contractions of one sweep)",
                   "peak_source": f"{pk_kind}: {peak_note}",
                   "work": "per sweep 4 o^2 v^2 R + 16 X v^2 R algorithmic flops"}
    dominant = roof_mttkrp if mttkrp_ms >= solve_ms else roof_solve
    line = {
        "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.precision,
        "data": "synthetic (seeded; shapes of the paper's molecules)",
        "config": {"workload": WORKLOAD, "o": O, "v": V, "X": XAUX, "R": RANK,
                   "precision": args.precision, "r_chunk": args.r_chunk,
                   "l2": "inputs larger than L2 (tau, B operand planes ~0.5 GB)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "mttkrp_tflops": mttkrp_tflops,
        "phase_ms": phases,
        "roofline": dominant,
        "roofline_mttkrp": roof_mttkrp,
        "roofline_solve": roof_solve,
        "precision_variants": variants,
        "fp64_gpu": {"ms_per_sweep": f64_ms, "sweeps_per_s": 1000.0 / f64_ms,
                     "speedup_mixed_vs_fp64": value / world / (1000.0 / f64_ms)},
        "accuracy": {"sweeps": n_cmp, "E_cp_mixed": E_mixed, "E_cp_fp64": E_f64,
                     "dE_kcal_per_mol": abs(E_mixed - E_f64) * KCAL,
                     "dE_rel": abs(E_mixed - E_f64) / abs(E_f64),
                     "meets_0.1_kcal": abs(E_mixed - E_f64) * KCAL <= 0.1, "E_exact": E_exact,
                     "mttkrp_rel_err": mttkrp_err(M_mixed),
                     "rank_error_kcal_per_mol": abs(E_f64 - E_exact) * KCAL,
                     "fit_mixed": fits_mixed[-1], "fit_fp64": fits_f64[-1]},
        "e2e": {"value": e2e_value, "unit": "sweeps/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "step": f"one warm-started solve of {SWEEPS_PER_SOLVE} sweeps: tau H2D, operand rebuild, sweeps, "
                        f"factors + fit history D2H"},
        "gpu_launches": int(st["kernels_per_sweep"]) * args.steps,
        "clocks": {k: ck[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "clock_samples": ck["samples"],
        "cpu_baseline": cpu,
        "fit_after_timed": fit_last,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_batch(args, world, rank, local):
    """64 uneven instances (o in [4,24], v in [40,240], X = 3v, R in [2v,4v]) swept
    together from one CUDA graph; one step = one sweep of every instance."""
    import numpy as np
    import torch
    from paper_2503_10380_gb300 import binding, inputs
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    shapes = inputs.batch_shapes(64, seed=SEED)
    data = [inputs.make_inputs_torch(*sh, seed=SEED + k, device=dev) for k, sh in enumerate(shapes)]
    flops = sum(alg_flops(*sh) for sh in shapes)
    probs = []
    for (B, tau, fac) in data:
        cp = binding.CpAls(B, tau, fac, precision=args.precision)
        cp.autotune()
        probs.append(cp)
    batch = binding.Batch(probs, nstreams=8)
    batch.sweep(args.warmup, want_fits=False)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    clocks = ClockSampler(local)
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    batch.sweep(args.steps, want_fits=False)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = reduce_max(e0.elapsed_time(e1), world, dev)
    launches = batch.kernels_per_sweep()
    # plain FP64 form of the same batch
    f64 = [binding.CpAls(B, tau, fac, precision="fp64") for (B, tau, fac) in data]
    fb = binding.Batch(f64, nstreams=8)
    fb.sweep(1, want_fits=False)
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    fb.sweep(2, want_fits=False)
    g1.record(stream)
    torch.cuda.synchronize()
    f64_ms = g0.elapsed_time(g1) / 2
    fb.close()
    for p in f64:
        p.close()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # oracle sweeps over the first instances until ~15 s, scaled by flops to the batch
        from oracle import ppl_oracle as orc
        t_or, fl_or, k = 0.0, 0.0, 0
        while t_or < 15.0 and k < len(shapes):
            B, tau, fac = data[k]
            o = shapes[k][0]
            Bvv = np.ascontiguousarray(B.cpu().numpy()[:, o:, o:])
            t = tau.cpu().numpy()
            t0 = time.perf_counter()
            orc.als_sweep(Bvv, t, fac, np.ones(shapes[k][3]))
            t_or += time.perf_counter() - t0
            fl_or += alg_flops(*shapes[k])
            k += 1
        cores, how = oracle_cores()
        cpu = {"value": (fl_or / flops) / t_or, "unit": "batch sweeps/s", "cores": cores, "kind": "oracle",
               "sample": f"one FP64 oracle sweep of each of the first {k} instances, scaled by flops to all 64; "
                         f"threads from {how}"}
    pk, pk_kind = peaks()
    peak, _ = tensor_peak(pk, args.precision)
    tflops = flops / (ms / args.steps / 1000.0) / 1e12
    value = world * args.steps / (ms / 1000.0)
    line = {
        "metric": METRIC, "value": value, "unit": "batch sweeps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.precision, "data": "synthetic (seeded; shapes of the paper's molecules)",
        "config": {"workload": "cp-als-ppl batch of 64 uneven instances (o 4-24, v 40-240, X = 3v, R 2v-4v), one graph",
                   "instances": 64, "precision": args.precision},
        "sweep_tflops": tflops,
        "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                     "traffic": None, "kernel": "whole batch sweep (MTTKRP flops / sweep time)",
                     "peak_source": f"{pk_kind}"},
        "fp64_gpu": {"ms_per_sweep": f64_ms, "speedup_mixed_vs_fp64": f64_ms / (ms / args.steps)},
        "gpu_launches": int(launches) * args.steps,
        "clocks": {k2: ck[k2] for k2 in ("sm_mhz", "sm_max_mhz", "reasons")},
        "cpu_baseline": cpu,
    }
    batch.close()
    for p in probs:
        p.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


PREC_CFG, PREC_SWEEPS = (40, 400, 1200, 1600), 20
SEQ_CFG, SEQ_STEPS, SEQ_MAX_SWEEPS, SEQ_EPS = (60, 600, 1800, 2400), 15, 50, 1e-6


def _factors_host(cp):
    return {k: t.cpu().numpy().copy() for k, t in cp.factors().items()}


def _timed_sweeps(cp, n, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cp.sweep(n, want_hist=False)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def run_precision(args, world, rank, local):
    """o=40 v=400 X=1200 R=1600: BF16x3, TF32 and TF32x3 against the plain FP64 GPU form
    from the same start after PREC_SWEEPS sweeps (energy in kcal/mol, relative
    error of every factor), and the sweep rate of each form."""
    import numpy as np
    import torch
    from paper_2503_10380_gb300 import binding, inputs
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    o, v, X, R = PREC_CFG
    B, tau, fac = inputs.make_inputs_torch(o, v, X, R, seed=SEED, device=dev)
    # ||R||^2 and E_exact from the TF32x3 tensor-core exact contraction (relative error ~1e-6)
    cp = binding.CpAls(B, tau, fac, precision="tf32x3")
    normR2, E_exact, _ = cp.exact_contract(mixed=True)
    cp.close()
    del cp
    f64 = binding.CpAls(B, tau, fac, precision="fp64")
    f64.set_normR2(normR2)
    f64.sweep(1, want_hist=False)
    torch.cuda.synchronize()
    f64_ms = _timed_sweeps(f64, PREC_SWEEPS - 1, stream)
    E64, F64, fit64 = f64.energy(), _factors_host(f64), f64.fit()
    f64.close()
    del f64
    torch.cuda.empty_cache()
    variants = {}
    clocks = None
    for prec in ("tf32x3", "bf16x3", "tf32"):
        cp = binding.CpAls(B, tau, fac, precision=prec, profile=True)
        rc_chosen = cp.autotune()
        cp.set_normR2(normR2)
        cp.sweep(PREC_SWEEPS, want_hist=False)
        E, F, fit = cp.energy(), _factors_host(cp), cp.fit()
        cp.sweep(args.warmup, want_hist=False)
        torch.cuda.synchronize()
        ck = ClockSampler(local) if prec == "tf32x3" else None
        ms = _timed_sweeps(cp, args.steps, stream)
        if ck is not None:
            clocks = ck.stop()
        acc = None
        for _ in range(3):
            cp.sweep(1, want_hist=False)
            ph = cp.phase_ms()
            acc = ph if acc is None else {k: acc[k] + ph[k] for k in acc}
        mt_ms = sum(acc[k] for k in ("tau_r", "chain_a", "chain_b", "s_and_p")) / 3
        launches = int(cp.stats()["kernels_per_sweep"])
        cp.close()
        del cp
        variants[prec] = {
            "ms_per_sweep": ms, "sweeps_per_s": 1000.0 / ms,
            "mttkrp_tflops": alg_flops(o, v, X, R) / (mt_ms / 1000.0) / 1e12,
            "speedup_vs_fp64_gpu": f64_ms / ms, "E_cp": E, "fit": fit,
            "dE_kcal_per_mol": abs(E - E64) * KCAL, "dE_rel": abs(E - E64) / abs(E64),
            "factor_rel_err": {m: float(np.linalg.norm(F[m] - F64[m]) / np.linalg.norm(F64[m])) for m in F64},
            "kernels_per_sweep": launches, "r_chunk": rc_chosen,
        }
    ms = reduce_max(variants["tf32x3"]["ms_per_sweep"], world, dev)
    pk, pk_kind = peaks()
    peak, peak_note = tensor_peak(pk, "tf32x3")
    tf = variants["tf32x3"]["mttkrp_tflops"]
    line = {
        "metric": METRIC, "value": world * 1000.0 / ms, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "tf32x3", "data": "synthetic (seeded; shapes of the paper's molecules)",
        "config": {"workload": f"cp-als-ppl precision study o={o} v={v} X={X} R={R}, {PREC_SWEEPS} sweeps "
                               f"from one start in FP64, BF16x3 and TF32", "o": o, "v": v, "X": X, "R": R,
                   "l2": "inputs larger than L2"},
        "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                     "traffic": None, "kernel": "all MTTKRP contractions of one sweep (phase events)",
                     "peak_source": f"{pk_kind}: {peak_note}"},
        "fp64_gpu": {"ms_per_sweep": f64_ms, "E_cp": E64, "fit": fit64},
        "variants": variants,
        "E_exact_tf32x3": E_exact, "normR2_tf32x3": normR2,
        "rank_error_kcal_per_mol": abs(E64 - E_exact) * KCAL,
        "gpu_launches": variants["tf32x3"]["kernels_per_sweep"] * args.steps,
        "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")} if clocks else None,
        "cpu_baseline": oracle_estimate(o, v, X, R) if rank == 0 and world == 1 and not args.no_cpu_baseline else None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_sequence(args, world, rank, local):
    """o=60 v=600 X=1800 R=2400: SEQ_STEPS CC-like steps tau_k = tau_{k-1} + dtau_k,
    each a CPD warm-started from the previous factors on the device and swept
    until |dfit| < SEQ_EPS (at most SEQ_MAX_SWEEPS sweeps); ||R_k||^2 from the
    tensor-core exact contraction at every step."""
    import torch
    from paper_2503_10380_gb300 import binding, inputs
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    o, v, X, R = SEQ_CFG
    B, tau, fac = inputs.make_inputs_torch(o, v, X, R, seed=SEED, device=dev)
    rms0 = float(torch.sqrt(torch.mean(tau * tau)))
    torch.cuda.empty_cache()
    cp = binding.CpAls(B, tau, fac, precision=args.precision, profile=True)
    rc_chosen = cp.autotune()
    clocks = ClockSampler(local)
    steps, t_solve, t_exact, n_sweeps = [], 0.0, 0.0, 0
    for k in range(SEQ_STEPS):
        if k > 0:
            tau += inputs.tau_increment_t(torch, rms0, tuple(tau.shape), k, seed=SEED, device=dev)
            cp.set_tau(tau)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        normR2, E_exact, _ = cp.exact_contract(mixed=True)
        t1 = time.perf_counter()
        sweeps, fits, _ = cp.solve(SEQ_MAX_SWEEPS, "dfit", SEQ_EPS)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        E = cp.energy()
        t_exact += t1 - t0
        t_solve += t2 - t1
        n_sweeps += sweeps
        steps.append({"k": k, "sweeps": sweeps, "stop": "dfit" if sweeps < SEQ_MAX_SWEEPS else "max_sweeps",
                      "fit": fits[sweeps - 1] if sweeps else None,
                      "dfit_last": abs(fits[sweeps - 1] - fits[sweeps - 2]) if sweeps > 1 else None,
                      "E_cp": E, "E_exact_mixed": E_exact, "solve_s": t2 - t1, "exact_s": t1 - t0})
        if rank == 0:
            print(json.dumps({"progress": steps[-1]}), file=sys.stderr, flush=True)
    ck = clocks.stop()
    acc = None
    for _ in range(3):
        cp.sweep(1, want_hist=False)
        ph = cp.phase_ms()
        acc = ph if acc is None else {kk: acc[kk] + ph[kk] for kk in acc}
    phases = {kk: acc[kk] / 3 for kk in acc}
    mt_ms = phases["tau_r"] + phases["chain_a"] + phases["chain_b"] + phases["s_and_p"]
    ms_sweep = _timed_sweeps(cp, 3, stream)
    launches = int(cp.stats()["kernels_per_sweep"])
    cp.close()
    del cp
    torch.cuda.empty_cache()
    f64 = binding.CpAls(B, tau, fac, precision="fp64")
    f64.sweep(1, want_hist=False)
    torch.cuda.synchronize()
    f64_ms = _timed_sweeps(f64, 1, stream)
    f64.close()
    t_solve = reduce_max(t_solve, world, dev)
    pk, pk_kind = peaks()
    peak, _ = tensor_peak(pk, args.precision)
    tf = alg_flops(o, v, X, R) / (mt_ms / 1000.0) / 1e12
    line = {
        "metric": METRIC, "value": world * n_sweeps / t_solve, "unit": "sweeps/s", "n_gpus": world,
        "steps": SEQ_STEPS, "warmup": 0, "ms_per_step": 1000.0 * t_solve / n_sweeps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
        "data": "synthetic (seeded; shapes of the paper's molecules)",
        "config": {"workload": f"cp-als-ppl warm-started CC-like sequence o={o} v={v} X={X} R={R}, {SEQ_STEPS} steps, "
                               f"|dfit| < {SEQ_EPS} or {SEQ_MAX_SWEEPS} sweeps", "o": o, "v": v, "X": X, "R": R,
                   "l2": "inputs larger than L2 (tau 10.4 GB)"},
        "sweeps_total": n_sweeps, "solve_s": t_solve, "exact_contract_s": t_exact, "r_chunk": rc_chosen,
        "ms_per_sweep_steady": ms_sweep, "phase_ms": phases,
        "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                     "traffic": None, "kernel": "all MTTKRP contractions of one sweep (phase events)",
                     "peak_source": f"{pk_kind}"},
        "fp64_gpu": {"ms_per_sweep": f64_ms, "speedup_mixed_vs_fp64": f64_ms / ms_sweep},
        "per_step": steps,
        "gpu_launches": launches * n_sweeps,
        "clocks": {kk: ck[kk] for kk in ("sm_mhz", "sm_max_mhz", "reasons")},
        "cpu_baseline": oracle_estimate(o, v, X, R) if rank == 0 and world == 1 and not args.no_cpu_baseline else None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["bf16x3", "tf32", "tf32x3"], default=None,
                    help="tensor-core precision of the MTTKRP (default: tf32x3, the split that meets the "
                         "0.1 kcal/mol bar; bf16x3 for --workload batch)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--r-chunk", type=int, default=0, help="rank columns per pass of the MTTKRP chain (0 = auto)")
    ap.add_argument("--workload", choices=["single", "batch", "precision", "sequence"], default="single",
                    help="single: o=20 v=200 X=600 R=800 (default); batch: 64 uneven instances; "
                         "precision: o=40 v=400 X=1200 R=1600 in FP64, BF16x3 and TF32; "
                         "sequence: o=60 v=600 X=1800 R=2400, 15 warm-started CC-like steps")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "bf16x3" if args.workload == "batch" else "tf32x3"
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup()
    if world > 1:
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        torch.distributed.init_process_group(backend=backend)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        elif args.workload == "batch":
            run_batch(args, world, rank, local)
        elif args.workload == "precision":
            run_precision(args, world, rank, local)
        elif args.workload == "sequence":
            run_sequence(args, world, rank, local)
        else:
            run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
