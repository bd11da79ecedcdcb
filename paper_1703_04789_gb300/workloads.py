"""Ready-made workloads and a profiling driver.

``hubbard_chain_handles`` prepares the L=24, D=256, n_beta=8 Hubbard workload (targets S=0 and
S=1) the way the benchmark does: seeded random MPS, GPU canonicalisation, warm-up sweeps,
checkpoint.  ``python -m paper_1703_04789_gb300.workloads --sweeps W --applies A`` runs the
warm-up sweeps and then A projected actions at the middle site of the optimised MPS, so that a
profiler can capture the block-GEMM launches of a converged state; with ``--profile-sweep`` it
also runs one more full sweep of the S=0 target inside the NVTX range ``profile_sweep`` (the
launches of every kernel kind of a sweep, for a launch list).
"""
from __future__ import annotations

import argparse

import numpy as np

HUBBARD_L24 = {"L": 24, "N": 24, "D": 256, "n_beta": 8, "U": 4.0, "targets": [[0, 0], [2, 2]], "seed": 2}


def hubbard_chain_handles(warm_sweeps: int, spec=HUBBARD_L24, targets=None, **opts):
    from . import Spmps, inputs
    out = []
    for twoM, twoS in (targets or spec["targets"]):
        labels, tens = inputs.random_mps(spec["L"], spec["N"], twoM, spec["D"], spec["seed"])
        dev = Spmps(spec["L"], spec["N"], twoM, twoS, spec["n_beta"], spec["D"], **opts)
        dev.set_hubbard(1.0, spec["U"])
        dev.set_mps(labels, tens, center=0)
        dev.canonicalize()
        energies, _ = dev.sweep(warm_sweeps) if warm_sweeps > 0 else (np.zeros(0), 0)
        out.append({"dev": dev, "twoM": twoM, "twoS": twoS, "ckpt": dev.get_mps(),
                    "e_warm": [float(e) for e in energies]})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sweeps", type=int, default=2)
    ap.add_argument("--applies", type=int, default=3)
    ap.add_argument("--site", type=int, default=11)
    ap.add_argument("--profile-sweep", action="store_true")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "tf32", "3xtf32"])
    args = ap.parse_args()
    import torch
    from . import build
    build.build()
    h = hubbard_chain_handles(args.sweeps, targets=[[0, 0]], autotune=args.autotune, precision=args.precision)[0]
    dev = h["dev"]
    lay = dev.x_layout(args.site)
    x = torch.tensor(np.random.default_rng(0).standard_normal(lay["n_x"]), device="cuda")
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    dev.apply_heff(args.site, x, y, z)  # environments and plan of the site, outside the range
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("profile_applies")
    for _ in range(args.applies):
        ms = dev.apply_heff_timed(args.site, x, y, z)
    torch.cuda.nvtx.range_pop()
    fl = dev.apply_flops(args.site)
    print({"n_x": lay["n_x"], "flops": fl.tolist(), "phase_ms": ms.tolist(),
           "gemm_tflops": float((fl[0] + fl[2]) / ((ms[1] + ms[3]) * 1e-3) / 1e12)})
    if args.profile_sweep:
        ck = dev.get_mps()
        dev.set_mps(*ck[:2], center=ck[2])
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("profile_sweep")
        E, _ = dev.sweep(1)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print({"profile_sweep_E": float(E[0]), "iterations": dev.davidson_stats()[0]})


if __name__ == "__main__":
    main()
