"""The metric-block Davidson correction on the GPU (precond = metric_block) against the oracle.

N_eff is block-diagonal in (N of the left bond index, n(s1), n(s2)); the correction solves with
the shifted blocks, t = (N_b + s I)^-1 r, and the converged x is replaced by the representative
(N + s I)^-1 N x before decimation (x is defined only modulo ker N_eff).  The lowest generalised
eigenvalue of a step (Eq. geproblem) does not depend on the correction, so theta is compared with
the oracle's solve from the same MPS.  Bounds: 1e-9 relative on theta from a converged solve
(|r| < 1e-9: the error of theta is quadratic in the residual).
"""
import numpy as np
import pytest

from oracle import fock, mpo as M, mps as S
from paper_1703_04789_gb300 import inputs
from tests.gpu_util import require_gpu


def _dev(L, N, twoM, twoS, D, G, U=4.0, **kw):
    from paper_1703_04789_gb300 import Spmps
    dev = Spmps(L, N, twoM, twoS, G, D, **kw)
    dev.set_hubbard(1.0, U)
    return dev


@pytest.mark.gpu
@pytest.mark.parametrize("case", [(6, 6, 0, 0, 12, 4, 3), (8, 8, 0, 0, 32, 5, 1), (7, 7, 1, 3, 20, 4, 2)])
def test_metric_block_step_theta_matches_oracle(case):
    require_gpu()
    L, N, twoM, twoS, D, G, seed = case
    labels, tens = inputs.random_mps(L, N, twoM, D, seed)
    P = S.prepare(labels, tens, M.hubbard_mpo(L, 1.0, 4.0), twoS, twoM, G)
    dev = _dev(L, N, twoM, twoS, D, G, precond="metric_block", dav_tol_r=1e-9, dav_max_iter=400)
    dev.set_mps(P.mps.labels, P.mps.A, center=0)
    th, it = dev.optimize_step(0, True)
    x0 = P.two_site(0)
    mask = S.two_site_mask(P.mps.labels[0], P.mps.labels[2])
    dh, dn = P.diagonal(0)
    res = S.davidson(lambda v: P.apply(v, 0), x0, dh, dn, mask, tol_r=1e-9, max_iter=400, precond="metric_block",
                     metric_blocks=P.metric_blocks(0))
    assert res.converged
    assert abs(th - res.theta) < 1e-9 * max(1.0, abs(res.theta)), (th, res.theta, it)
    dev.close()


@pytest.mark.gpu
def test_shared_state_sweep_theta_at_every_step():
    """L=8, D=32, n_beta=5 (truncating): after two warm-up sweeps, at every step of the third the
    GPU's current MPS is handed to the oracle, both solve Eq. geproblem at that step and theta must
    agree; then the GPU takes the step (Davidson, decimation, environment update) and the next
    step starts from its MPS.  Both solve to |r| < 1e-7: with the metric inverted down to N-norms
    of 1e-7 the residual has a noise floor near 1e-8 here, and theta from |r| < 1e-7 agrees with
    the |r| < 1e-8 value to under 1e-9 (measured with the oracle on this workload)."""
    require_gpu()
    L, N, twoM, twoS, D, G = 8, 8, 0, 0, 32, 5
    labels, tens = inputs.random_mps(L, N, twoM, D, 1)
    dev = _dev(L, N, twoM, twoS, D, G, precond="metric_block", dav_tol_r=1e-7, dav_max_iter=600)
    dev.set_mps(labels, tens, center=0)
    dev.canonicalize()
    dev.sweep(2)
    mpo = M.hubbard_mpo(L, 1.0, 4.0)
    checked = 0
    for k, mr in S.sweep_schedule(L):
        lab, ts, c = dev.get_mps()
        P = S.Projected(S.MPS([np.asarray(q) for q in lab], [np.asarray(t) for t in ts], c), mpo, twoS, twoM, G)
        P.build_left(k)
        P.build_right(k + 2)
        x0 = P.two_site(k)
        mask = S.two_site_mask(P.mps.labels[k], P.mps.labels[k + 2])
        dh, dn = P.diagonal(k)
        res = S.davidson(lambda v: P.apply(v, k), x0, dh, dn, mask, tol_r=1e-7, max_iter=600,
                         precond="metric_block", metric_blocks=P.metric_blocks(k))
        th, it = dev.optimize_step(k, mr, allow_not_converged=True)
        assert res.converged and it < 600, (k, mr, it, res.iterations)
        assert abs(th - res.theta) < 1e-9 * max(1.0, abs(res.theta)), (k, mr, th, res.theta)
        checked += 1
    assert checked == 2 * L - 3
    dev.close()


@pytest.mark.gpu
def test_metric_block_sweeps_need_fewer_iterations_and_reach_lower_energy():
    """From the same checkpoint (L=10, D=48, n_beta=6, after two sweeps with the diagonal
    correction): one sweep with the metric-block correction takes well under half the Davidson
    iterations of one with the diagonal correction and ends at an energy no higher."""
    require_gpu()
    L, N, D, G = 10, 10, 48, 6
    labels, tens = inputs.random_mps(L, N, 0, D, 2)
    dev = _dev(L, N, 0, 0, D, G)
    dev.set_mps(labels, tens, center=0)
    dev.canonicalize()
    dev.sweep(2)
    ck = dev.get_mps()
    dev.close()
    out = {}
    for pc in ("diag", "metric_block"):
        d = _dev(L, N, 0, 0, D, G, precond=pc)
        d.set_mps(*ck[:2], center=ck[2])
        E, _ = d.sweep(1)
        out[pc] = (float(E[0]), d.davidson_stats()[0])
        d.close()
    assert out["metric_block"][1] < 0.5 * out["diag"][1], out
    assert out["metric_block"][0] <= out["diag"][0] + 1e-8, out


@pytest.mark.gpu
@pytest.mark.parametrize("case", [(6, 6, 0, 0, 64, 4), (5, 5, 1, 3, 32, 3)])
def test_metric_block_untruncated_sweeps_reach_exact_spin_state(case):
    require_gpu()
    L, N, twoM, twoS, D, G = case
    h1, eri = inputs.hubbard_chain(L, 1.0, 4.0)
    Na, Nb = inputs.electron_counts(N, twoM)
    e_ed, _, _ = fock.lowest_spin_state(L, Na, Nb, h1, eri, twoS)
    labels, tens = inputs.random_mps(L, N, twoM, D, 1)
    dev = _dev(L, N, twoM, twoS, D, G, precond="metric_block", dav_tol_r=1e-8)
    dev.set_mps(labels, tens, center=0)
    dev.canonicalize()
    E, st = dev.sweep(3)
    assert abs(E[-1] - e_ed) < 1e-8, (E, e_ed)
    s = 0.5 * twoS
    assert abs(dev.expect_s2() - s * (s + 1)) < 1e-8
    dev.close()
