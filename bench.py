#!/usr/bin/env python3
"""Benchmark of the SP-MPS hot path on GB300 (one JSON line on rank 0).

Workload: open Hubbard chain L=24, t=1, U=4, half filling, D=256, n_beta=8 Gauss-Legendre
points, targets S=0 (2M=0) and S=1 (2M=2).  Set-up (untimed): seeded random (N, M)-symmetric MPS,
GPU canonicalisation, W warm-up two-site sweeps (which also harvest training pairs for the
learned Davidson correction), checkpoint, training of the correction.

One step = for each target, restore the checkpoint (untimed) and run one full two-site sweep
(2K-3 steps of generalised Davidson with the projected H_eff/N_eff action, decimation to D,
environment updates: every row of the hot path) in the fast form: all beta points and blocks in
grouped launches with autotuned GEMM tiles, the H part of the block products in 3xTF32 on the
tensor cores until the Davidson residual is below 1e-5, then FP64.  Beside it, from the same
checkpoints: the FP64 plain form (one launch per beta point and phase, fixed tiles) for both
targets, and the all-FP64 fast form and the fast form with the learned correction for the S=0
target, each with its energy difference to the plain form.

Value = target-sweeps per second of the fast form (both targets' sweeps over their device time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (plain float64 NumPy) on the host cores on a bounded
sample of the same workload: one projected action per step, scaled to a sweep by the number of
actions per sweep of the FP64 plain form.  N > 1 (under torchrun) runs independent replicas.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SP-MPS sweep time & projected H_eff·x TFLOP/s vs FP64 plain at 1e-6 Eh"
# Projected actions per sweep of the FP64 plain form on this workload (measured on GB300, mean of
# the two targets); scales the oracle's per-action time to a sweep for --impl reference.
ACTIONS_PER_PLAIN_SWEEP = 5745
# DRAM bytes per k_gemm_oz launch of the middle-site FP64 action (phase A 73.1 MB, phase C 131.2 MB,
# ncu dram__bytes_read.sum + dram__bytes_write.sum of the current kernel, Hubbard L=24, D=256, sites
# (11, 12) after one warm-up sweep)
TRAFFIC_PER_LAUNCH = 102.2e6
# FP16 digit products per FP64 multiply-add in the split-product GEMM (levels 2..9 of 7 x 7 digits)
DIGIT_PRODUCTS = 34
WORKLOAD = {
    "workload": "Hubbard chain L=24 open, t=1, U=4, N=24, targets (2M,2S)=(0,0) and (2,2), D=256, "
                "n_beta=8; step = one two-site sweep per target from a checkpoint taken after the warm-up sweeps",
    "L": 24, "N": 24, "D": 256, "n_beta": 8, "U": 4.0, "targets": [[0, 0], [2, 2]], "site": 11,
    "mps": "seeded random (N,M)-symmetric MPS, inputs.random_mps(seed=2), canonicalised on the GPU",
    "davidson": "|r| < 1e-6 and |dtheta| < 1e-10, subspace 20, cap 200",
    "forms": {"fast": "grouped launches over all beta points and blocks, autotuned GEMM tiles, H part of the "
                      "block products in 3xTF32 on the tensor cores (stacked tcgen05 GEMM) until |r| < 1e-5, then "
                      "FP64; every FP64 block product of the action (N_eff x, the FP64 finish) as exact 8-bit digit "
                      "products on the tensor cores (split-product GEMM, FP64-accurate); diagonal correction",
              "fast_fp64_tc": "fast with every block product of the action FP64-accurate on the split-product GEMM "
                              "(no 3xTF32 stage)",
              "fast_fp64": "fast with every block product in FP64 on the FP64 pipe (no tensor cores)",
              "fast_mma_sync": "fast with the warp-level mma.sync kernel for the 3xTF32 stage",
              "fp64_plain": "one launch per beta point and phase, fixed tiles, FP64, diagonal correction",
              "fast_learned": "fast with the learned Davidson correction"},
    "l2": "flushed before every timed sweep (256 MiB write); environments of all bonds exceed L2",
}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    return rank, world


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 8 for i in range(4) if r[4 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def max_over_ranks(ms: float, device) -> float:
    """The slowest rank's time (replicas run independently; the job is done when all are)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, max_ms: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    return units_per_rank * world / (max_ms * 1e-3)


def _setup(args):
    """Checkpoints after the warm-up sweeps (batched FP64 form, harvesting training pairs for the
    learned correction) and the trained correction; returns per-target dicts and its parameters."""
    from paper_1703_04789_gb300.workloads import hubbard_chain_handles
    hs = hubbard_chain_handles(0, batched=True)
    for h in hs:
        dev = h["dev"]
        dev.mlp_harvest(True, samples_per_iteration=256, capacity=1 << 22)
        e, _ = dev.sweep(args.warmup)
        dev.mlp_harvest(False)
        h["e_warm"] = [float(v) for v in e]
        h["ckpt"] = dev.get_mps()
        h["ckpt_bytes"] = int(sum(t.size for t in h["ckpt"][1]) * 8)
    # one correction for both targets, trained on the pairs harvested by the first target
    X, _ = hs[0]["dev"].mlp_data()
    X1, _ = hs[1]["dev"].mlp_data()
    l0, l1 = hs[0]["dev"].mlp_train(600, batch=4096, lr=1e-3, seed=5)
    params = hs[0]["dev"].mlp_get_params()
    info = {"pairs": int(X.shape[0] + X1.shape[0]), "pairs_used": int(X.shape[0]), "loss_first": l0, "loss_last": l1}
    for h in hs:
        h["dev"].close()
        del h["dev"]
    return hs, params, info


def _time_sweeps(dev, ckpt, steps, flush, torch):
    stream = torch.cuda.ExternalStream(dev.stream_handle())
    out = {"ms": [], "E": [], "iters": [], "refine_iters": [], "status": []}
    for _ in range(steps):
        dev.set_mps(*ckpt[:2], center=ckpt[2])
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        E, st = dev.sweep(1)
        e1.record(stream)
        e1.synchronize()
        out["ms"].append(e0.elapsed_time(e1))
        out["E"].append(float(E[0]))
        out["status"].append(int(st))
        it, rit = dev.davidson_stats()
        out["iters"].append(it)
        out["refine_iters"].append(rit)
    return out


FORMS = {
    "fast": dict(batched=True, autotune=True, precision="3xtf32", precond="diag", fp64_tensor_cores=True),
    "fp64_plain": dict(batched=False, autotune=False, precision="fp64", precond="diag"),
    "fast_fp64_tc": dict(batched=True, autotune=True, precision="fp64", precond="diag", fp64_tensor_cores=True),
    "fast_fp64": dict(batched=True, autotune=True, precision="fp64", precond="diag"),
    "fast_learned": dict(batched=True, autotune=True, precision="3xtf32", precond="learned", fp64_tensor_cores=True),
    "fast_mma_sync": dict(batched=True, autotune=True, precision="3xtf32", precond="diag",
                          tensor_core_kernel="mma_sync", fp64_tensor_cores=True),
}


def _handle(form, twoM, twoS, params=None):
    from paper_1703_04789_gb300 import Spmps
    W = WORKLOAD
    dev = Spmps(W["L"], W["N"], twoM, twoS, W["n_beta"], W["D"], **FORMS[form])
    dev.set_hubbard(1.0, W["U"])
    if FORMS[form]["precond"] == "learned":
        dev.mlp_set_params(params)
    return dev


def run_ours(args):
    import torch
    rank, world = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    from paper_1703_04789_gb300 import build as B, device_fp64_peak, device_tf32_peak
    B.build()
    hs, params, mlp_info = _setup(args)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    key = lambda h: f"2S={h['twoS']}"

    # the headline form: the contract's timed steps, both targets (no per-launch profiler)
    fast = [_handle("fast", h["twoM"], h["twoS"]) for h in hs]
    launches0 = sum(d.stats()["launches"] for d in fast)
    flops0 = [d.stats()["apply_flops_total"] for d in fast]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    res_fast = [_time_sweeps(d, h["ckpt"], args.steps, flush, torch) for d, h in zip(fast, hs)]
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    launches = sum(d.stats()["launches"] for d in fast) - launches0
    apply_flops = sum(d.stats()["apply_flops_total"] - f0 for d, f0 in zip(fast, flops0))
    total_ms = max_over_ranks(sum(sum(r["ms"]) for r in res_fast), "cuda")
    value = whole_job_rate(args.steps * len(hs), world, total_ms)

    # kernel breakdown from a separate, untimed sweep of the S=0 target with the per-launch profiler
    names = ["gemm_fp64", "comb", "ritz", "davidson_vector_ops", "decimation_eigen", "host_planning",
             "metric_factor", "metric_solve", "gemm_tensor_core", "gemm_fp64_split"]
    fast[0].profile(True)
    prof_run = _time_sweeps(fast[0], hs[0]["ckpt"], 1, flush, torch)
    breakdown = {}
    for kind, name in enumerate(names):
        st = fast[0].kernel_stats(kind)
        breakdown[name] = {"ms": round(st["ms"], 2), "launches": int(st["launches"]), "flops": st["flops"]}
    fast[0].profile(False)
    breakdown["profiled_sweep_ms"] = round(prof_run["ms"][0], 2)

    # end to end through the host C ABI: checkpoint upload (host -> device), sweep, energy read-back
    t0 = time.perf_counter()
    for d, h in zip(fast, hs):
        d.set_mps(*h["ckpt"][:2], center=h["ckpt"][2])
        d.sweep(1)
    e2e_s = max_over_ranks((time.perf_counter() - t0) * 1e3, "cuda") * 1e-3
    e2e_value = len(hs) * world / e2e_s
    # the block GEMMs at the middle site of the S=0 target, from the fast form's checkpointed MPS:
    # phases A and C of the H part alone (the fast form's 3xTF32 products, y only) and of the whole
    # FP64-accurate action (y and z) on the split-product GEMM and on the FP64 pipe (CUDA events on
    # the handle's stream, warm, mean of 5)
    site = WORKLOAD["site"]

    def middle_site_phases(dev, with_z):
        lay = dev.x_layout(site)
        xs = torch.tensor(np.random.default_rng(0).standard_normal(lay["n_x"]), device="cuda")
        ys = torch.empty_like(xs)
        zs = torch.empty_like(xs) if with_z else None
        dev.apply_heff(site, xs, ys, zs)
        torch.cuda.synchronize()
        ph = np.mean([dev.apply_heff_timed(site, xs, ys, zs) for _ in range(5)], axis=0)
        return ph, dev.apply_costs(site)

    for d in fast:
        d.close()
    dtc = _handle("fast", hs[0]["twoM"], hs[0]["twoS"])
    dtc.set_mps(*hs[0]["ckpt"][:2], center=hs[0]["ckpt"][2])
    phase_tc, (fl_op, by_op) = middle_site_phases(dtc, with_z=False)
    dtc.close()
    doz = _handle("fast_fp64_tc", hs[0]["twoM"], hs[0]["twoS"])
    doz.set_mps(*hs[0]["ckpt"][:2], center=hs[0]["ckpt"][2])
    phase_oz, _ = middle_site_phases(doz, with_z=True)
    doz.close()
    d64 = _handle("fast_fp64", hs[0]["twoM"], hs[0]["twoS"])
    d64.set_mps(*hs[0]["ckpt"][:2], center=hs[0]["ckpt"][2])
    phase, _ = middle_site_phases(d64, with_z=True)
    d64.close()

    # the FP64 plain form (one sweep per target) and the mixed-precision / learned variants
    # (one sweep of the S=0 target), all from the same checkpoints
    res_plain = []
    for h in hs:
        d = _handle("fp64_plain", h["twoM"], h["twoS"])
        res_plain.append(_time_sweeps(d, h["ckpt"], 1, flush, torch))
        d.close()
    variants = {}
    for form in ("fast_fp64_tc", "fast_fp64", "fast_mma_sync", "fast_learned"):
        d = _handle(form, hs[0]["twoM"], hs[0]["twoS"], params)
        r = _time_sweeps(d, hs[0]["ckpt"], 1, flush, torch)
        d.close()
        variants[form] = {"sweep_s": round(r["ms"][0] / 1e3, 4), "E": r["E"][0], "iters": r["iters"][0],
                          "fp64_refinement_iters": r["refine_iters"][0],
                          "abs_dE_vs_fp64_plain": abs(r["E"][0] - res_plain[0]["E"][0])}

    peak = device_fp64_peak(torch.cuda.current_device())
    tf32_peaks = (device_tf32_peak(0), device_tf32_peak(1))
    hbm = _measured_peaks().get("hbm_gbs")
    if rank != 0:
        return
    fast_mean = {key(h): statistics.mean(r["ms"]) / 1e3 for h, r in zip(hs, res_fast)}
    plain_s = {key(h): r["ms"][0] / 1e3 for h, r in zip(hs, res_plain)}
    dE = max(abs(a - r2["E"][0]) for r1, r2 in zip(res_fast, res_plain) for a in r1["E"])
    line = {
        "metric": METRIC, "value": round(value, 6), "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 (H block products 3xTF32 until |r| < 1e-5, then FP64-accurate split products)", "data": "synthetic",
        "config": dict(WORKLOAD, parallelism="replicas" if world > 1 else "single"),
        "sweep_s": {"fast": {k: round(v, 4) for k, v in fast_mean.items()},
                    "fp64_plain": {k: round(v, 4) for k, v in plain_s.items()}},
        "speedup_vs_fp64_plain": round(sum(plain_s.values()) / sum(fast_mean.values()), 3),
        "energies": {"fast": {key(h): r["E"] for h, r in zip(hs, res_fast)},
                     "fp64_plain": {key(h): r["E"] for h, r in zip(hs, res_plain)},
                     "max_abs_dE": dE, "within_1e-6": dE <= 1e-6},
        "davidson_iterations_per_sweep": {"fast": {key(h): r["iters"] for h, r in zip(hs, res_fast)},
                                          "fp64_plain": {key(h): r["iters"] for h, r in zip(hs, res_plain)}},
        "iterations_after_fp64_switch": {"fast": {key(h): r["refine_iters"] for h, r in zip(hs, res_fast)}},
        "steps_at_iteration_cap": {"fast": {key(h): r["status"] for h, r in zip(hs, res_fast)}},
        "variants_2S=0": variants,
        "learned_correction": mlp_info,
        "apply_tflops": round(apply_flops / (total_ms * 1e-3) / 1e12, 6),
        "roofline": _roofline(phase_oz, phase_tc, phase, fl_op, by_op, hbm, tf32_peaks, peak, breakdown,
                              _measured_peaks().get("bf16_tflops")),
        "time_breakdown_ms": dict(breakdown, timed_sweeps_total_ms=round(total_ms, 2)),
        "e2e": {"value": round(e2e_value, 6), "unit": "sweeps/s", "h2d_bytes_per_step": sum(h["ckpt_bytes"] for h in hs),
                "d2h_bytes_per_step": 8 * len(hs)},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        actions = statistics.mean(r["iters"][0] for r in res_plain)
        line["cpu_baseline"] = cpu_baseline_sample(actions_per_sweep=actions)
    print(json.dumps(line), flush=True)


def _measured_peaks():
    """The driver's measured peaks (HBM copy GB/s, cuBLAS BF16 TFLOP/s); {} when absent."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _roofline(phase_oz, phase_tc, phase64, fl_op, by_op, hbm, tf32_peaks, fp64_peak, breakdown, f16_peak):
    """Roofline of the fast form's dominant kernel and of its other block-GEMM kernels.

    The kernel breakdown of a fast sweep (separate profiled pass) puts the split-product GEMM first
    (k_gemm_oz: every FP64-accurate block product of phases A and C, H and N).  Its arithmetic is
    FP16 tensor-core MMAs, DIGIT_PRODUCTS digit products per FP64 multiply-add, so its roofline is
    the FP16 dense tensor peak (the measured BF16 burst; FP16 has the same nominal dense rate):
    achieved = DIGIT_PRODUCTS x the algorithmic FP64 flops of phases A and C of the middle-site action
    / their CUDA-event time.  Beside it, the same algorithmic FP64 flops per second against the
    measured FP64 pipe (what an FP64 GEMM could reach), the FP64 pipe kernel on the same action, and
    the 3xTF32 products of the H part (k_gemm_tc) against the HBM bandwidth and the tcgen05
    kind::tf32 peak."""
    flops64 = float(fl_op[0][0] + fl_op[0][2] + fl_op[1][0] + fl_op[1][2])
    t_oz = (phase_oz[1] + phase_oz[3]) * 1e-3
    t64 = (phase64[1] + phase64[3]) * 1e-3
    t_tc = (phase_tc[1] + phase_tc[3]) * 1e-3
    bytes_tc = float(by_op[0][0] + by_op[0][2])
    flops_tc = float(fl_op[0][0] + fl_op[0][2])
    peak_bw = hbm if hbm else 6800.0
    peak16 = f16_peak if f16_peak else 1900.0
    goz = breakdown.get("gemm_fp64_split", {})
    g64 = breakdown.get("gemm_fp64", {})
    gtc = breakdown.get("gemm_tensor_core", {})
    total = breakdown.get("profiled_sweep_ms") or 0.0
    ach_oz = DIGIT_PRODUCTS * flops64 / t_oz / 1e12
    fp64_eq = flops64 / t_oz / 1e12
    ach64 = flops64 / t64 / 1e12
    return {
        "bound": "tensor",
        "kernel": "k_gemm_oz: FP64-accurate split-product GEMM (tcgen05 kind::f16 on 8-bit digits), phases A and C "
                  "of the projected action (H and N) at sites (11, 12), S=0",
        "achieved": round(ach_oz, 4), "peak": round(peak16, 1), "unit": "TFLOP/s",
        "frac": round(ach_oz / peak16, 5),
        "peak_source": ("measured cuBLAS BF16 burst (MEASURED_PEAKS.json bf16_tflops) as the FP16 dense peak "
                        "(same nominal rate)") if f16_peak else "fallback 1.9 PFLOP/s",
        "achieved_note": f"{DIGIT_PRODUCTS} FP16 digit products per algorithmic FP64 multiply-add",
        "traffic": TRAFFIC_PER_LAUNCH,
        "traffic_note": "dram bytes read + written per k_gemm_oz launch (mean of the phase-A and phase-C launches) "
                        "from one ncu capture of the middle-site action",
        "phase_ms": [round(float(v), 4) for v in phase_oz],
        "share_of_fast_sweep": round(goz.get("ms", 0.0) / total, 4) if total else None,
        "fp64_equivalent": {"achieved_tflops": round(fp64_eq, 4), "fp64_pipe_peak_tflops": round(fp64_peak, 4),
                            "frac_of_fp64_pipe": round(fp64_eq / fp64_peak, 4) if fp64_peak else None,
                            "peak_source": "measured: FP64 FMA-chain kernel on all SMs (spmps_device_fp64_peak)"},
        "fp64_pipe_kernel": {
            "kernel": "k_gemm_f64 on the same action (the fast_fp64 form)", "bound": "alu",
            "achieved_tflops": round(ach64, 4), "peak_tflops": round(fp64_peak, 4),
            "frac": round(ach64 / fp64_peak, 4) if fp64_peak else None,
            "phase_ms": [round(float(v), 4) for v in phase64],
            "share_of_fast_sweep": round(g64.get("ms", 0.0) / total, 4) if total else None},
        "tensor_core_kernel": {
            "kernel": "k_gemm_tc: stacked tcgen05 kind::tf32 (3xTF32) H products of phases A and C, same site",
            "bound": "hbm", "achieved_GBs": round(bytes_tc / t_tc / 1e9, 2), "peak_GBs": round(peak_bw, 1),
            "frac": round(bytes_tc / t_tc / 1e9 / peak_bw, 4),
            "peak_source": "measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if hbm else "fallback 6800 GB/s",
            "algorithmic_bytes": bytes_tc, "phase_ms": [round(float(v), 4) for v in phase_tc],
            "achieved_tflops": round(flops_tc / t_tc / 1e12, 4),
            "peak_tflops_tcgen05_tf32": round(tf32_peaks[1], 1), "peak_tflops_mma_sync_tf32": round(tf32_peaks[0], 1),
            "tensor_frac": round(flops_tc / t_tc / 1e12 / tf32_peaks[1], 5) if tf32_peaks[1] else None,
            "share_of_fast_sweep": round(gtc.get("ms", 0.0) / total, 4) if total else None,
            "note": "algorithmic flops (one product per multiply-add; the 3xTF32 split is not counted)"},
    }


def _oracle_setup(twoM=0, twoS=0):
    from oracle import mpo as M, mps as S
    from paper_1703_04789_gb300 import inputs
    W = WORKLOAD
    labels, tens = inputs.random_mps(W["L"], W["N"], twoM, W["D"], 2)
    mps = S.MPS([l.copy() for l in labels], [t.copy() for t in tens], 0)
    P = S.Projected(mps, M.hubbard_mpo(W["L"], 1.0, W["U"]), twoS, twoM, W["n_beta"])
    k = W["site"]
    P.build_right(k + 2)
    P.build_left(k)
    ql, qr = mps.labels[k], mps.labels[k + 2]
    x = np.where(S.two_site_mask(ql, qr), np.random.default_rng(11).standard_normal((ql.shape[0], 4, 4, qr.shape[0])), 0.0)
    return P, x


def cpu_baseline_sample(actions_per_sweep: float):
    """The oracle as it stands: one projected action of the S=0 target on the host cores, scaled to
    a sweep by the number of actions per sweep (Davidson iterations of the FP64 plain form)."""
    P, x = _oracle_setup()
    t0 = time.perf_counter()
    P.apply(x, WORKLOAD["site"])
    dt = time.perf_counter() - t0
    return {"value": 1.0 / (dt * actions_per_sweep), "unit": "sweeps/s", "cores": os.cpu_count(), "kind": "oracle",
            "seconds_per_action": round(dt, 3), "actions_per_sweep": round(actions_per_sweep, 1),
            "sample": "one projected action (y and z, 8 beta points) of the S=0 target at sites (11,12), dense NumPy "
                      "float64 with BLAS on all host cores, environments built untimed; sweep time estimated as "
                      "time per action x actions per FP64-plain sweep (environment updates and decimation not "
                      "counted, so the estimate favours the oracle)"}


def run_reference(args):
    rank, world = _dist()
    if rank != 0:
        return
    P, x = _oracle_setup()
    for _ in range(args.warmup):
        P.apply(x, WORKLOAD["site"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        P.apply(x, WORKLOAD["site"])
    dt = time.perf_counter() - t0
    per_action = dt / args.steps
    value = 1.0 / (per_action * ACTIONS_PER_PLAIN_SWEEP)
    line = {
        "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(per_action * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": dict(WORKLOAD, step_note="reference step = one projected action of the S=0 target (bounded "
                                           "sample), scaled to a sweep by ACTIONS_PER_PLAIN_SWEEP"),
        "cpu_baseline": {"value": value, "unit": "sweeps/s", "kind": "oracle", "cores": os.cpu_count(),
                         "sample": "one projected action of the S=0 target per step, dense NumPy float64, scaled by "
                                   f"{ACTIONS_PER_PLAIN_SWEEP} actions per sweep"},
        "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _alg_flops_cpu() -> float:
    """Algorithmic flops of one projected action of the S=0 target, counted from the block
    structure alone (same rule as the library planner: 2*m*n*k per symmetry-allowed block
    product and 2*rows*cols per MPO-leg term)."""
    from oracle import mpo as M
    from oracle.quadrature import projector_quadrature, site_rotation
    from paper_1703_04789_gb300 import inputs
    W = WORKLOAD
    return float(_count_apply_flops(inputs.mps_structure(W["L"], W["N"], 0, W["D"]), W["site"],
                                    M.hubbard_mpo(W["L"], 1.0, W["U"]), W["n_beta"], 0, 0))


def _count_apply_flops(struct, k, mpo, G, twoS, twoM):
    import numpy as _np
    from oracle.mpo import rotate_mpo, identity_mpo
    from oracle.quadrature import projector_quadrature
    LN, LM = (0, 1, 1, 2), (0, -1, 1, 0)
    bl = {(n, m): d for n, m, d in struct[k]}
    br = {(n, m): d for n, m, d in struct[k + 2]}

    def groups(b):
        g = {}
        for (n, m), d in b.items():
            g[n] = g.get(n, 0) + d
        return g
    gl, gr = groups(bl), groups(br)
    beta, c = projector_quadrature(twoS, twoM, G)
    total = 0.0
    for ops in (mpo, identity_mpo(len(mpo))):
        # channel charges
        cn = [[0]]
        for W in ops:
            nxt = [0] * W.shape[1]
            for a in range(W.shape[0]):
                for b in range(W.shape[1]):
                    nz = _np.argwhere(W[a, b] != 0)
                    if len(nz):
                        s, t = nz[0]
                        nxt[b] = cn[-1][a] + LN[s] - LN[t]
            cn.append(nxt)
        cnl, cnr = cn[k], cn[k + 2]
        for g in range(G):
            Wr = rotate_mpo(ops, beta[g])
            W1, W2 = Wr[k], Wr[k + 1]
            WW = _np.einsum("wvst,vuij->wusitj", W1, W2).reshape(W1.shape[0], W2.shape[1], 16, 16)
            # phase A
            for (na, ma), da in bl.items():
                wid = sum(br.get((na + LN[s1] + LN[s2], ma + LM[s1] + LM[s2]), 0) for s1 in range(4) for s2 in range(4))
                if wid == 0:
                    continue
                for w in range(len(cnl)):
                    Ga = gl.get(na + cnl[w], 0)
                    total += 2.0 * Ga * da * wid
            # phase B
            for u in range(len(cnr)):
                for nG, dG in gl.items():
                    n0 = nG - cnr[u]
                    for s in range(16):
                        nb = n0 + LN[s >> 2] + LN[s & 3]
                        if nb not in gr:
                            continue
                        nterm = 0
                        for w in range(len(cnl)):
                            if nG - cnl[w] not in gl:
                                continue
                            for t in range(16):
                                if WW[w, u, s, t] != 0 and (nG - cnl[w] + LN[t >> 2] + LN[t & 3]) in gr:
                                    nterm += 1
                        total += 2.0 * dG * gr[nb] * nterm
            # phase C
            for (na, ma), da in bl.items():
                for s in range(16):
                    qb = (na + LN[s >> 2] + LN[s & 3], ma + LM[s >> 2] + LM[s & 3])
                    if qb not in br:
                        continue
                    for u in range(len(cnr)):
                        nbp = qb[0] - cnr[u]
                        if nbp in gr:
                            total += 2.0 * da * br[qb] * gr[nbp]
    return total


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
