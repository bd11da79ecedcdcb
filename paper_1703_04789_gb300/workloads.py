"""Ready-made workloads and a profiling driver.

``hubbard_chain_handles`` prepares the L=24, D=256, n_beta=8 Hubbard workload (targets S=0 and
S=1) the way the benchmark does: seeded random MPS, GPU canonicalisation, warm-up sweeps,
checkpoint.  ``ab_initio_action`` runs one projected action of the K=20, N=30, 2M=2S=10,
n_beta=12 active-space workload at a given bond dimension (``--ab-initio-D 100 200``).  ``python -m paper_1703_04789_gb300.workloads --sweeps W --applies A`` runs the
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


AB_INITIO_K20 = {"K": 20, "N": 30, "twoM": 10, "twoS": 10, "n_beta": 12, "seed": 3}
# the same integrals and electron count with M = 0 and target S = 0 (a projector that removes the
# S = 1 .. 5 components, where the high-spin target above keeps all of M = S = 5)
AB_INITIO_K20_S0 = {"K": 20, "N": 30, "twoM": 0, "twoS": 0, "n_beta": 12, "seed": 3}


def ab_initio_action(D: int, spec=AB_INITIO_K20, precisions=("fp64", "3xtf32", "fp64_tc"), site=None, m_screen=0.0):
    """One projected action at the middle of the synthetic active-space workload (K=20, N=30,
    2M=2S=10, n_beta=12; integrals from inputs.synthetic_active_space) for a seeded random MPS of
    bond dimension D, canonicalised on the GPU: per precision form the phase times (CUDA events),
    the algorithmic flops and bytes, the error of y against the FP64 action, and the device memory
    in use (environments of every bond, the action's intermediates).  Form "fp64_tc" is the FP64
    action with its block products of phases A and C split into exact digit products on the
    tensor cores (fp64_tensor_cores)."""
    import torch
    from . import Spmps, inputs
    K, N, twoM, twoS, G = spec["K"], spec["N"], spec["twoM"], spec["twoS"], spec["n_beta"]
    h1, eri, ecore = inputs.synthetic_active_space(K, spec["seed"])
    labels, tens = inputs.random_mps(K, N, twoM, D, spec["seed"])
    k = K // 2 - 1 if site is None else site
    out = {"K": K, "N": N, "twoM": twoM, "twoS": twoS, "n_beta": G, "D": D, "site": k, "m_screen": m_screen,
           "forms": {}}
    y64 = None
    for prec in precisions:
        dev = Spmps(K, N, twoM, twoS, G, D, precision="fp64" if prec == "fp64_tc" else prec, autotune=False,
                    m_screen=m_screen, fp64_tensor_cores=prec == "fp64_tc")
        dev.set_hamiltonian(h1, eri, ecore)
        dev.set_mps(labels, tens, center=0)
        dev.canonicalize()
        lay = dev.x_layout(k)
        x = torch.tensor(np.random.default_rng(1).standard_normal(lay["n_x"]), device="cuda")
        y, z = torch.empty_like(x), torch.empty_like(x)
        dev.apply_heff(k, x, y, z)
        torch.cuda.synchronize()
        free, total = torch.cuda.mem_get_info()
        ms = np.mean([dev.apply_heff_timed(k, x, y, z) for _ in range(2)], axis=0)
        fl, by = dev.apply_costs(k)
        yv = y.cpu().numpy()
        if prec == "fp64":
            y64 = yv
        out["forms"][prec] = {"n_x": lay["n_x"], "phase_ms": [round(float(v), 4) for v in ms],
                              "flops": fl.tolist(), "bytes": by.tolist(),
                              "device_memory_used_GB": round((total - free) / 1e9, 2),
                              "rel_err_y_vs_fp64": None if y64 is None else float(np.abs(yv - y64).max() / np.abs(y64).max())}
        dev.close()
        torch.cuda.synchronize()
    return out


def ab_initio_step(D: int, spec=AB_INITIO_K20, forms=("fp64", "3xtf32_tc", "fp64_tc"), site=None, max_iter=200):
    """One two-site optimisation step (Davidson to |r| < 1e-6 and decimation to D) at the middle of
    the synthetic active-space workload, from the same canonicalised random MPS, per form: wall
    time of the step (environments of the site built before it), Davidson iterations and theta,
    with |theta - theta_fp64|.  Forms: "fp64" (FP64 pipe), "fp64_tc" (every block product of
    phases A and C FP64-accurate on the split-product GEMM), "3xtf32_tc" (3xTF32 H products until
    |r| < 1e-5, FP64-accurate split products otherwise)."""
    import time
    import torch
    from . import Spmps, inputs
    K, N, twoM, twoS, G = spec["K"], spec["N"], spec["twoM"], spec["twoS"], spec["n_beta"]
    h1, eri, ecore = inputs.synthetic_active_space(K, spec["seed"])
    labels, tens = inputs.random_mps(K, N, twoM, D, spec["seed"])
    k = K // 2 - 1 if site is None else site
    out = {"K": K, "N": N, "twoM": twoM, "twoS": twoS, "n_beta": G, "D": D, "site": k, "steps": {}}
    opts = {"fp64": dict(precision="fp64"), "fp64_tc": dict(precision="fp64", fp64_tensor_cores=True),
            "3xtf32_tc": dict(precision="3xtf32", fp64_tensor_cores=True)}
    # canonical form with the centre on site k: canonicalise, then steps 0 .. k-1 with one Davidson
    # iteration each (the Ritz vector of a one-vector basis is the current two-site tensor, so the
    # decimation only moves the gauge)
    g = Spmps(K, N, twoM, twoS, G, D, dav_max_iter=1, fp64_tensor_cores=True)
    g.set_hamiltonian(h1, eri, ecore)
    g.set_mps(labels, tens, center=0)
    g.canonicalize()
    for j in range(k):
        g.optimize_step(j, True, allow_not_converged=True)
    ck = g.get_mps()
    g.close()
    th64 = None
    for form in forms:
        dev = Spmps(K, N, twoM, twoS, G, D, dav_max_iter=max_iter, **opts[form])
        dev.set_hamiltonian(h1, eri, ecore)
        dev.set_mps(*ck[:2], center=ck[2])
        lay = dev.x_layout(k)
        x = torch.zeros(lay["n_x"], dtype=torch.float64, device="cuda")
        dev.apply_heff(k, x, torch.empty_like(x), torch.empty_like(x))  # environments and plan of the site
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        th, it = dev.optimize_step(k, True, allow_not_converged=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if form == "fp64":
            th64 = th
        out["steps"][form] = {"seconds": round(dt, 3), "iterations": int(it), "theta": float(th),
                              "abs_dtheta_vs_fp64": None if th64 is None else abs(th - th64)}
        print(form, out["steps"][form], flush=True)
        dev.close()
        torch.cuda.synchronize()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--ab-initio-D", type=int, nargs="*", default=None,
                    help="one action of the K=20 active-space workload at each of these bond dimensions")
    ap.add_argument("--ab-initio-step", type=int, nargs="*", default=None,
                    help="one two-site step of the K=20 active-space workload at each of these bond dimensions")
    ap.add_argument("--step-forms", nargs="*", default=["fp64", "3xtf32_tc", "fp64_tc"])
    ap.add_argument("--singlet", action="store_true", help="the K=20 workload with 2M = 2S = 0")
    ap.add_argument("--sweeps", type=int, default=2)
    ap.add_argument("--applies", type=int, default=3)
    ap.add_argument("--site", type=int, default=11)
    ap.add_argument("--profile-sweep", action="store_true")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "tf32", "3xtf32"])
    ap.add_argument("--fp64-tensor-cores", action="store_true",
                    help="FP64 block products of the action as exact digit products on the tensor cores")
    args = ap.parse_args()
    import torch
    from . import build
    build.build()
    if args.ab_initio_D or args.ab_initio_step:
        import json
        spec = AB_INITIO_K20_S0 if args.singlet else AB_INITIO_K20
        for D in args.ab_initio_D or []:
            print(json.dumps(ab_initio_action(D, spec=spec)), flush=True)
        for D in args.ab_initio_step or []:
            print(json.dumps(ab_initio_step(D, spec=spec, forms=tuple(args.step_forms))), flush=True)
        return
    h = hubbard_chain_handles(args.sweeps, targets=[[0, 0]], autotune=args.autotune, precision=args.precision,
                              fp64_tensor_cores=args.fp64_tensor_cores)[0]
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
