"""Host logic of bench.py that needs no GPU: the roofline record built from phase times, costs and
peaks (units, the FP64-equivalent rate, shares of the profiled sweep)."""
import numpy as np

import bench


def test_roofline_record_from_phase_times():
    fl = np.array([[4.0e8, 1.0e8, 6.0e8], [2.0e8, 0.5e8, 3.0e8]])  # per op: phases A, B, C
    by = np.array([[1.0e8, 2.0e7, 3.0e8], [5.0e7, 1.0e7, 1.5e8]])
    ph_oz = [0.01, 0.5, 0.1, 0.5]  # zero fill, A, B, C in ms
    ph_tc = [0.01, 0.2, 0.1, 0.2]
    ph_64 = [0.01, 1.0, 0.1, 1.0]
    bd = {"gemm_fp64_split": {"ms": 300.0}, "gemm_fp64": {"ms": 10.0}, "gemm_tensor_core": {"ms": 100.0},
          "profiled_sweep_ms": 1000.0}
    r = bench._roofline(ph_oz, ph_tc, ph_64, fl, by, 6000.0, (300.0, 1200.0), 1.25, bd, 2000.0)
    flops64 = 4.0e8 + 6.0e8 + 2.0e8 + 3.0e8
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - bench.DIGIT_PRODUCTS * flops64 / 1.0e-3 / 1e12) < 1e-3
    assert abs(r["frac"] - r["achieved"] / 2000.0) < 1e-5
    assert abs(r["fp64_equivalent"]["achieved_tflops"] - flops64 / 1.0e-3 / 1e12) < 1e-4
    assert abs(r["fp64_pipe_kernel"]["achieved_tflops"] - flops64 / 2.0e-3 / 1e12) < 1e-4
    assert r["share_of_fast_sweep"] == 0.3
    tc = r["tensor_core_kernel"]
    assert abs(tc["achieved_GBs"] - (1.0e8 + 3.0e8) / 0.4e-3 / 1e9) < 1e-2
    assert tc["share_of_fast_sweep"] == 0.1
    assert r["traffic"] == bench.TRAFFIC_PER_LAUNCH
