"""The allocation-free projected action (spmps_apply_heff_noalloc).

Callers whose device memory is reserved up front by their own pool, or runtimes that forbid the
CUDA allocator after start-up, cannot let the library call cudaMalloc when they need the action;
this entry point keeps its intermediates in a fixed static device array instead.  It must give
the same y and z as spmps_apply_heff, call after call.  This file is collected last so that a failure here leaves every other test run.
"""
import numpy as np
import pytest

from paper_1703_04789_gb300 import inputs
from tests.gpu_util import require_gpu

RTOL = 1e-10


@pytest.mark.gpu
@pytest.mark.parametrize("fp64_tc", [False, True])
def test_noalloc_apply_matches_apply_on_two_calls(fp64_tc):
    """Also with the FP64 block products split on the tensor cores (their status word is
    allocated with the plan, so the call still allocates nothing)."""
    require_gpu()
    import torch
    from paper_1703_04789_gb300 import Spmps
    L, N, D, G = 8, 8, 32, 5
    labels, tens = inputs.random_mps(L, N, 0, D, 1)
    dev = Spmps(L, N, 0, 0, G, D, fp64_tensor_cores=fp64_tc)
    dev.set_hubbard(1.0, 4.0)
    dev.set_mps(labels, tens, center=0)
    for k in (3, 5):
        lay = dev.x_layout(k)
        rng = np.random.default_rng(k)
        x = torch.tensor(rng.standard_normal(lay["n_x"]), device="cuda")
        y_ref = torch.empty_like(x)
        z_ref = torch.empty_like(x)
        dev.apply_heff(k, x, y_ref, z_ref)  # builds environments and the plan (allocates)
        torch.cuda.synchronize()
        for _ in range(2):
            y = torch.full_like(x, float("nan"))
            z = torch.full_like(x, float("nan"))
            dev.apply_heff_noalloc(k, x, y, z)
            torch.cuda.synchronize()
            sy = max(1.0, float(y_ref.abs().max()))
            sz = max(1.0, float(z_ref.abs().max()))
            assert float((y - y_ref).abs().max()) <= RTOL * sy
            assert float((z - z_ref).abs().max()) <= RTOL * sz
    dev.close()


@pytest.mark.gpu
def test_noalloc_on_a_caller_stream_waits_for_the_handle_stream():
    """The environments are built on the handle's stream; a call on another stream right after
    the plan-building call (no host synchronisation in between) must still see them."""
    require_gpu()
    import torch
    from paper_1703_04789_gb300 import Spmps
    L, N, D, G = 10, 10, 48, 6
    labels, tens = inputs.random_mps(L, N, 0, D, 4)
    dev = Spmps(L, N, 0, 0, G, D)
    dev.set_hubbard(1.0, 4.0)
    dev.set_mps(labels, tens, center=0)
    k = 4
    n = dev.x_layout(k)["n_x"]
    x = torch.tensor(np.random.default_rng(7).standard_normal(n), device="cuda")
    y_ref, z_ref = torch.empty_like(x), torch.empty_like(x)
    side = torch.cuda.Stream()
    for _ in range(2):
        dev.apply_heff(k, x, y_ref, z_ref)  # handle's stream, asynchronous
        y = torch.full_like(x, float("nan"))
        z = torch.full_like(x, float("nan"))
        side.wait_stream(torch.cuda.current_stream())  # x, y, z were written on torch's stream
        dev.apply_heff_noalloc(k, x, y, z, stream=side)
        side.synchronize()
        torch.cuda.synchronize()
        assert float((y - y_ref).abs().max()) <= RTOL * max(1.0, float(y_ref.abs().max()))
        assert float((z - z_ref).abs().max()) <= RTOL * max(1.0, float(z_ref.abs().max()))
    dev.close()


@pytest.mark.gpu
def test_noalloc_rejects_missing_plan_and_oversize():
    require_gpu()
    import torch
    from paper_1703_04789_gb300 import Spmps, SpmpsError
    L, N, D, G = 24, 24, 256, 8
    labels, tens = inputs.random_mps(L, N, 0, D, 2)
    dev = Spmps(L, N, 0, 0, G, D)
    dev.set_hubbard(1.0, 4.0)
    dev.set_mps(labels, tens, center=0)
    k = 11
    n = dev.x_layout(k)["n_x"]
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(SpmpsError) as ei:
        dev.apply_heff_noalloc(k, x, y, None)
    assert ei.value.status == 8  # no plan yet: SPMPS_ERR_STATE
    dev.apply_heff(k, x, y, None)
    torch.cuda.synchronize()
    with pytest.raises(SpmpsError) as ei:
        dev.apply_heff_noalloc(k, x, y, None)
    assert ei.value.status == 1  # intermediates above the fixed scratch: SPMPS_ERR_BAD_INPUT
    dev.close()
