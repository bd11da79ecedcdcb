"""Approximate M-sector screening (Sec. 2.3.1, closing paragraph; spmps_options.m_screen) on the GPU
against the oracle's screened action, and its error against the exact action.

The screened action is a definition of its own: per operator, beta point and channel, the block
products whose environment sub-block between a bra label and a ket label is below tau times the
largest such sub-block of the channel are dropped.  The GPU and the oracle apply the same rule, so
the screened y and z agree to FP64 rounding (1e-10 relative to max |y|); the error of the screened
action against the exact one is reported and must shrink with tau.
"""
import numpy as np
import pytest

from oracle import mpo as M, mps as S
from paper_1703_04789_gb300 import inputs
from tests.gpu_util import masked_random_two_site, require_gpu


@pytest.mark.gpu
@pytest.mark.parametrize("tau", [1e-4, 1e-2])
def test_screened_action_matches_oracle_every_site(tau):
    require_gpu()
    from paper_1703_04789_gb300 import Spmps
    L, N, D, G = 8, 8, 32, 5
    labels, tens = inputs.random_mps(L, N, 0, D, 1)
    P = S.prepare(labels, tens, M.hubbard_mpo(L, 1.0, 4.0), 0, 0, G)
    P.build_left(L - 2)
    dev = Spmps(L, N, 0, 0, G, D, m_screen=tau)
    dev.set_hubbard(1.0, 4.0)
    dev.set_mps(P.mps.labels, P.mps.A, center=0)
    ref = Spmps(L, N, 0, 0, G, D)
    ref.set_hubbard(1.0, 4.0)
    ref.set_mps(P.mps.labels, P.mps.A, center=0)
    rng = np.random.default_rng(5)
    for k in range(L - 1):
        ql, qr = P.mps.labels[k], P.mps.labels[k + 2]
        x = masked_random_two_site(ql, qr, rng)
        y_ref, z_ref = P.apply(x, k, screen=tau)
        lay = dev.x_layout(k)
        yv, zv = dev.apply_heff_host(k, dev.pack(x, lay, ql, qr))
        y, z = dev.unpack(yv, lay, ql, qr), dev.unpack(zv, lay, ql, qr)
        assert np.abs(y - y_ref).max() <= 1e-10 * max(1.0, np.abs(y_ref).max()), k
        assert np.abs(z - z_ref).max() <= 1e-10 * max(1.0, np.abs(z_ref).max()), k
        assert dev.apply_flops(k).sum() <= ref.apply_flops(k).sum()
    dev.close()
    ref.close()


@pytest.mark.gpu
def test_screening_error_and_work_against_the_exact_action():
    """L=24, D=256, n_beta=8, middle site of a random canonical MPS: the relative error of the
    screened y against the exact one grows with tau while the algorithmic flops fall."""
    require_gpu()
    from paper_1703_04789_gb300 import Spmps
    L, N, D, G = 24, 24, 256, 8
    labels, tens = inputs.random_mps(L, N, 0, D, 2)
    k = 11
    out = []
    y0 = None
    for tau in (0.0, 1e-6, 1e-4, 1e-2):
        dev = Spmps(L, N, 0, 0, G, D, m_screen=tau)
        dev.set_hubbard(1.0, 4.0)
        dev.set_mps(labels, tens, center=0)
        dev.canonicalize()
        n = dev.x_layout(k)["n_x"]
        x = np.random.default_rng(3).standard_normal(n)
        y, z = dev.apply_heff_host(k, x)
        fl = float(dev.apply_flops(k).sum())
        dev.close()
        if y0 is None:
            y0, fl0 = y, fl
        out.append((tau, float(np.abs(y - y0).max() / np.abs(y0).max()), fl / fl0))
    print("screening (tau, max rel error of y, flops fraction):", out)
    errs = [e for _, e, _ in out]
    flops = [f for _, _, f in out]
    assert errs[0] == 0.0 and flops[0] == 1.0
    assert errs[1] <= errs[2] <= errs[3] and flops[3] <= flops[2] <= flops[1] <= 1.0
    assert errs[1] < 1e-4
