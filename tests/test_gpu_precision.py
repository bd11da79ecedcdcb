"""Reduced-precision forms of the projected action (TF32 and 3xTF32 tensor-core block products
for H_eff x, FP32 accumulation) and the FP64 refinement that restores the energy.

Bounds: TF32 keeps 10 mantissa bits (unit roundoff 2^-11 ~ 4.9e-4 per product), so the action is
compared at 1e-2 relative to max |y|; 3xTF32 recovers about FP32 products (2^-24 ~ 6e-8 each,
FP32 accumulation over reductions of a few hundred terms), compared at 1e-5.  z (N_eff x) stays
FP64 and must be identical.  After refinement the Davidson eigenvalue must equal the FP64 one
to 1e-9 relative.
"""
import numpy as np
import pytest

from oracle import mpo as M, mps as S
from paper_1703_04789_gb300 import inputs
from tests.gpu_util import require_gpu


def _dev(L, N, twoM, twoS, D, G, **kw):
    from paper_1703_04789_gb300 import Spmps
    d = Spmps(L, N, twoM, twoS, G, D, **kw)
    d.set_hubbard(1.0, 4.0)
    return d


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("tf32", 1e-2), ("3xtf32", 1e-5)])
def test_reduced_precision_action_within_bound(prec, tol):
    require_gpu()
    L, N, D, G = 10, 10, 48, 6
    labels, tens = inputs.random_mps(L, N, 0, D, 3)
    ref = _dev(L, N, 0, 0, D, G)
    fast = _dev(L, N, 0, 0, D, G, precision=prec)
    for d in (ref, fast):
        d.set_mps(labels, tens, center=0)
    for k in (0, 4, 8):
        n = ref.x_layout(k)["n_x"]
        x = np.random.default_rng(k).standard_normal(n)
        y0, z0 = ref.apply_heff_host(k, x)
        y1, z1 = fast.apply_heff_host(k, x)
        assert np.array_equal(z0, z1)
        err = np.abs(y1 - y0).max() / np.abs(y0).max()
        assert err < tol, (k, err)
        assert err > 0.0  # the tensor-core path really ran
    ref.close()
    fast.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["tf32", "3xtf32"])
def test_refined_theta_matches_fp64(prec):
    require_gpu()
    L, N, D, G = 8, 8, 32, 5
    labels, tens = inputs.random_mps(L, N, 0, D, 1)
    P = S.prepare(labels, tens, M.hubbard_mpo(L, 1.0, 4.0), 0, 0, G)
    out = {}
    for p in ("fp64", prec):
        d = _dev(L, N, 0, 0, D, G, precision=p, dav_tol_r=1e-8)
        d.set_mps(P.mps.labels, P.mps.A, center=0)
        out[p] = d.optimize_step(0, True)
        d.close()
    assert abs(out[prec][0] - out["fp64"][0]) < 1e-9 * max(1.0, abs(out["fp64"][0])), out


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["tf32", "3xtf32"])
def test_mixed_precision_sweeps_match_fp64(prec):
    """Whole sweeps with the reduced-precision action in the first Davidson stage (autotuned
    tiles, pre-split tensor-core operands, environments updated along the way): at D above the
    exact Schmidt rank both forms reach the same exact singlet energy, and every solve finishes
    in FP64."""
    require_gpu()
    from paper_1703_04789_gb300 import Spmps
    L, N, D, G = 8, 8, 256, 5
    labels, tens = inputs.random_mps(L, N, 0, D, 4)
    out = {}
    for p in ("fp64", prec):
        dev = Spmps(L, N, 0, 0, G, D, precision=p, autotune=True)
        dev.set_hubbard(1.0, 4.0)
        dev.set_mps(labels, tens, center=0)
        dev.canonicalize()
        E, _ = dev.sweep(3)
        out[p] = E
        if p != "fp64":
            it, refine = dev.davidson_stats()
            assert refine > 0
        dev.close()
    assert abs(out[prec][-1] - out["fp64"][-1]) < 1e-8, (out[prec], out["fp64"])
