#!/usr/bin/env python3
"""Benchmark of the SP-MPS hot path on GB300 (one JSON line on rank 0).

Workload: open Hubbard chain L=24, t=1, U=4, half filling, D=256, n_beta=8 Gauss-Legendre
points, targets S=0 (2M=0) and S=1 (2M=2).  Set-up (untimed): seeded random (N, M)-symmetric MPS,
canonicalised on the GPU, W warm-up two-site sweeps, checkpoint.  One step = for each target,
restore the checkpoint (untimed) and run one full two-site sweep (2K-3 steps of generalised
Davidson with the projected H_eff/N_eff action, decimation to D, environment updates): every row
of the hot path.  Value = algorithmic TFLOP/s of the projected actions issued in the timed sweeps
over the sweep time (symmetry-allowed block products only); sweep seconds are reported beside.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (plain float64 NumPy) on the host cores on a bounded
sample of the same workload (one projected action per step).  N > 1 (under torchrun) runs
independent replicas.
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
WORKLOAD = {
    "workload": "Hubbard chain L=24 open, t=1, U=4, N=24, targets (2M,2S)=(0,0) and (2,2), D=256, "
                "n_beta=8; step = one two-site sweep per target from a checkpoint taken after the warm-up sweeps",
    "L": 24, "N": 24, "D": 256, "n_beta": 8, "U": 4.0, "targets": [[0, 0], [2, 2]], "site": 11,
    "mps": "seeded random (N,M)-symmetric MPS, inputs.random_mps(seed=2), canonicalised on the GPU",
    "davidson": "diagonal preconditioner, |r| < 1e-6 and |dtheta| < 1e-10, subspace 20, cap 200",
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


def _setup_handles(args):
    from paper_1703_04789_gb300 import Spmps, inputs
    W = WORKLOAD
    handles = []
    for twoM, twoS in W["targets"]:
        labels, tens = inputs.random_mps(W["L"], W["N"], twoM, W["D"], 2)
        dev = Spmps(W["L"], W["N"], twoM, twoS, W["n_beta"], W["D"])
        dev.set_hubbard(1.0, W["U"])
        dev.set_mps(labels, tens, center=0)
        dev.canonicalize()
        e_warm, _ = dev.sweep(args.warmup)
        ckpt = dev.get_mps()
        handles.append({"dev": dev, "ckpt": ckpt, "twoS": twoS, "e_warm": [float(e) for e in e_warm],
                        "ckpt_bytes": int(sum(t.size for t in ckpt[1]) * 8)})
    return handles


def run_ours(args):
    import torch
    rank, world = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    from paper_1703_04789_gb300 import build as B, device_fp64_peak
    B.build()
    handles = _setup_handles(args)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    streams = [torch.cuda.ExternalStream(h["dev"].stream_handle()) for h in handles]
    launches0 = sum(h["dev"].stats()["launches"] for h in handles)
    flops0 = [h["dev"].stats()["apply_flops_total"] for h in handles]
    for h in handles:
        h["dev"].profile(True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sweep_ms = [[] for _ in handles]
    energies = [[] for _ in handles]
    iters = [[] for _ in handles]
    for _ in range(args.steps):
        for hi, h in enumerate(handles):
            dev = h["dev"]
            dev.set_mps(*h["ckpt"][:2], center=h["ckpt"][2])
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(streams[hi])
            E, st = dev.sweep(1)
            e1.record(streams[hi])
            e1.synchronize()
            sweep_ms[hi].append(e0.elapsed_time(e1))
            energies[hi].append(float(E[0]))
            iters[hi].append(dev.stats()["davidson_iterations"])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    gemm = [h["dev"].kernel_stats(0) for h in handles]
    comb = [h["dev"].kernel_stats(1) for h in handles]
    for h in handles:
        h["dev"].profile(False)
    launches = sum(h["dev"].stats()["launches"] for h in handles) - launches0
    apply_flops = sum(h["dev"].stats()["apply_flops_total"] - f0 for h, f0 in zip(handles, flops0))
    total_ms = sum(sum(m) for m in sweep_ms)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = apply_flops * world / (total_ms * 1e-3) / 1e12

    # end to end through the host C ABI: checkpoint upload (host -> device), sweep, energy read-back
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 2))):
        t0 = time.perf_counter()
        for h in handles:
            h["dev"].set_mps(*h["ckpt"][:2], center=h["ckpt"][2])
            h["dev"].sweep(1)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    per_step_flops = apply_flops / args.steps
    e2e_value = per_step_flops * len(e2e_ms) * world / (sum(e2e_ms) * 1e-3) / 1e12
    h2d = sum(h["ckpt_bytes"] for h in handles)
    d2h = 8 * len(handles)

    g_ms = sum(g["ms"] for g in gemm)
    g_fl = sum(g["flops"] for g in gemm)
    g_n = sum(g["launches"] for g in gemm)
    achieved = g_fl / (g_ms * 1e-3) / 1e12 if g_ms > 0 else 0.0
    peak = device_fp64_peak(torch.cuda.current_device())
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": round(value, 6), "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(WORKLOAD, parallelism="replicas" if world > 1 else "single"),
        "sweep_s": {f"2S={h['twoS']}": round(statistics.mean(m) / 1e3, 4) for h, m in zip(handles, sweep_ms)},
        "davidson_iterations_per_sweep": {f"2S={h['twoS']}": it for h, it in zip(handles, iters)},
        "energies": {f"2S={h['twoS']}": [round(e, 10) for e in E] for h, E in zip(handles, energies)},
        "roofline": {"bound": "alu", "kernel": "k_gemm_f64 (all block GEMMs of the sweep)",
                     "achieved": round(achieved, 6), "peak": round(peak, 6), "unit": "TFLOP/s",
                     "frac": round(achieved / peak, 4) if peak else None,
                     "peak_source": "measured: FP64 FMA-chain kernel on all SMs (nominal 1.25)",
                     "traffic": None, "launches": g_n, "avg_launch_ms": round(g_ms / max(1, g_n), 5),
                     "share_of_sweep": round(g_ms / total_ms, 4) if total_ms else None},
        "comb_kernel": {"launches": sum(c["launches"] for c in comb), "ms": round(sum(c["ms"] for c in comb), 3)},
        "e2e": {"value": round(e2e_value, 6), "unit": "TFLOP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(flops_per_apply=_alg_flops_cpu())
    print(json.dumps(line), flush=True)


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


def cpu_baseline_sample(flops_per_apply: float):
    """The oracle as it stands, one projected action of the S=0 target on the host cores."""
    P, x = _oracle_setup()
    t0 = time.perf_counter()
    P.apply(x, WORKLOAD["site"])
    dt = time.perf_counter() - t0
    return {"value": round(flops_per_apply / dt / 1e12, 9), "unit": "TFLOP/s", "cores": os.cpu_count(),
            "kind": "oracle", "seconds": round(dt, 3),
            "sample": "one projected action (y and z, 8 beta points) of the S=0 target at sites (11,12); "
                      "dense NumPy float64, BLAS threads = all host cores; environments built untimed"}


def run_reference(args):
    rank, world = _dist()
    if rank != 0:
        return
    from paper_1703_04789_gb300 import Spmps  # noqa: F401  (flop count of the same plan needs no GPU)
    flops = _alg_flops_cpu()
    P, x = _oracle_setup()
    for _ in range(args.warmup):
        P.apply(x, WORKLOAD["site"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        P.apply(x, WORKLOAD["site"])
    dt = time.perf_counter() - t0
    value = flops * args.steps / dt / 1e12
    line = {
        "metric": METRIC, "value": round(value, 9), "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": dict(WORKLOAD, step_note="reference step = the S=0 target's action only (bounded sample)"),
        "cpu_baseline": {"value": round(value, 9), "unit": "TFLOP/s", "kind": "oracle", "cores": os.cpu_count(),
                         "sample": "one projected action of the S=0 target per step, dense NumPy float64"},
        "e2e": {"value": round(value, 9), "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
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
    ap.add_argument("--steps", type=int, default=3)
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
