"""The C-ABI library builds for sm_103a, loads, and exports every entry point declared in
include/spmps.h; argument validation happens before any device work (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

from tests.gpu_util import gpu_available, library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "spmps.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(spmps_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    path = library()
    lib = C.CDLL(path)
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_bad_inputs_rejected_without_device_work():
    from paper_1703_04789_gb300 import Spmps, SpmpsError
    library()
    bad = [
        (1, 2, 0, 0, 4, 8),      # K < 2
        (4, 3, 0, 1, 4, 8),      # N + 2M odd
        (4, 4, 2, 0, 4, 8),      # 2S < |2M|
        (4, 4, 0, 1, 4, 8),      # 2S + N odd
        (4, 9, 1, 1, 4, 8),      # N > 2K
        (4, 4, 0, 0, 0, 8),      # n_beta < 1
        (4, 4, 0, 0, 4, 0),      # D < 1
        (4, 6, 6, 6, 4, 8),      # N_alpha = 6 > K
    ]
    for args in bad:
        with pytest.raises(SpmpsError) as ei:
            Spmps(*args)
        assert ei.value.status == 1, args
    for kw in ({"dav_max_iter": 0}, {"dav_max_sub": 3}, {"metric_max_dim": -1}, {"tc_wait_polls": -2}):
        with pytest.raises(SpmpsError) as ei:
            Spmps(4, 4, 0, 0, 2, 8, **kw)
        assert ei.value.status == 1, kw


@pytest.mark.parametrize("precond", ["diag", "metric", "learned", "olsen", "metric_block"])
def test_every_correction_option_passes_validation(precond):
    """Valid options are never rejected as bad input (without a GPU the create call then stops at
    the device with SPMPS_ERR_CUDA)."""
    from paper_1703_04789_gb300 import Spmps, SpmpsError
    library()
    try:
        Spmps(4, 4, 0, 0, 2, 8, precond=precond, metric_max_dim=64, tc_wait_polls=10).close()
    except SpmpsError as e:
        assert e.status != 1, e


def test_no_silent_fallback_without_gpu():
    if gpu_available():
        pytest.skip("a GPU is present")
    from paper_1703_04789_gb300 import Spmps, SpmpsError
    library()
    with pytest.raises(SpmpsError) as ei:
        Spmps(4, 4, 0, 0, 2, 8)
    assert ei.value.status == 6  # SPMPS_ERR_CUDA


@pytest.mark.parametrize("field,value", [("fp64_tensor_cores", 2), ("fp64_tensor_cores", -1),
                                         ("tensor_core_kernel", 2), ("precision", 3), ("m_screen", 1.5),
                                         ("precond", 5)])
def test_out_of_range_options_are_bad_input(field, value):
    """Options outside their documented ranges are refused by spmps_create before any device work."""
    import paper_1703_04789_gb300 as P
    lib = P.load_library(library())
    o = P.Options()
    lib.spmps_default_options(C.byref(o))
    setattr(o, field, value)
    h = C.c_void_p()
    assert lib.spmps_create(4, 4, 0, 0, 2, 8, C.byref(o), C.byref(h)) == 1
