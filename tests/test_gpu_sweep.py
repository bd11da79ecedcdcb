"""Davidson, decimation and sweeps on the GPU against the oracle and exact diagonalisation.

The lowest generalised eigenvalue theta of one two-site step (Eq. geproblem) is unique, so it
is compared between the CUDA path and the oracle from the same MPS; MPS tensors are not
compared (the eigenvector is defined only up to the kernel of N_eff).  Untruncated sweeps must
reach the lowest spin-S ED eigenvalue (independent of the projector), and <S^2> = S(S+1).
"""
import numpy as np
import pytest

from oracle import fock, mpo as M, mps as S, quadrature as Q
from paper_1703_04789_gb300 import inputs
from tests.gpu_util import require_gpu


def _dev(L, N, twoM, twoS, D, G, U=4.0, **kw):
    from paper_1703_04789_gb300 import Spmps
    dev = Spmps(L, N, twoM, twoS, G, D, **kw)
    dev.set_hubbard(1.0, U)
    return dev


@pytest.mark.gpu
@pytest.mark.parametrize("case", [(6, 6, 0, 0, 12, 4, 3), (8, 8, 0, 0, 32, 5, 1), (7, 7, 1, 3, 20, 4, 2)])
def test_step_theta_matches_oracle(case):
    require_gpu()
    L, N, twoM, twoS, D, G, seed = case
    labels, tens = inputs.random_mps(L, N, twoM, D, seed)
    P = S.prepare(labels, tens, M.hubbard_mpo(L, 1.0, 4.0), twoS, twoM, G)
    dev = _dev(L, N, twoM, twoS, D, G, dav_tol_r=1e-9, dav_max_iter=400)
    dev.set_mps(P.mps.labels, P.mps.A, center=0)
    th, it = dev.optimize_step(0, True)
    x0 = P.two_site(0)
    mask = S.two_site_mask(P.mps.labels[0], P.mps.labels[2])
    dh, dn = P.diagonal(0)
    res = S.davidson(lambda v: P.apply(v, 0), x0, dh, dn, mask, tol_r=1e-9, max_iter=400)
    assert res.converged
    assert abs(th - res.theta) < 1e-9 * max(1.0, abs(res.theta)), (th, res.theta, it)
    dev.close()


@pytest.mark.gpu
@pytest.mark.parametrize("case", [(4, 4, 0, 0, 16, 2), (4, 4, 2, 2, 16, 3), (6, 6, 0, 0, 64, 4), (5, 5, 1, 3, 32, 3)])
def test_untruncated_gpu_sweeps_reach_exact_spin_state(case):
    require_gpu()
    L, N, twoM, twoS, D, G = case
    h1, eri = inputs.hubbard_chain(L, 1.0, 4.0)
    Na, Nb = inputs.electron_counts(N, twoM)
    e_ed, _, _ = fock.lowest_spin_state(L, Na, Nb, h1, eri, twoS)
    labels, tens = inputs.random_mps(L, N, twoM, D, 1)
    dev = _dev(L, N, twoM, twoS, D, G, dav_tol_r=1e-8)
    dev.set_mps(labels, tens, center=0)
    dev.canonicalize()
    E, st = dev.sweep(4)
    assert abs(E[-1] - e_ed) < 1e-8, (E, e_ed)
    E2, nP = dev.energy()
    assert abs(E2 - e_ed) < 1e-8 and 0.0 < nP <= 1.0 + 1e-12
    s = 0.5 * twoS
    assert abs(dev.expect_s2() - s * (s + 1)) < 1e-8
    dev.close()


@pytest.mark.gpu
def test_canonicalize_preserves_the_functional():
    require_gpu()
    L, N, twoM, twoS, D, G = 8, 8, 0, 0, 24, 5
    labels, tens = inputs.random_mps(L, N, twoM, D, 5)
    P = S.prepare(labels, tens, M.hubbard_mpo(L, 1.0, 4.0), twoS, twoM, G)
    E_ref, nP_ref = P.energy(0)
    dev = _dev(L, N, twoM, twoS, D, G)
    dev.set_mps(labels, tens, center=0)
    dev.canonicalize()
    E, nP = dev.energy()
    assert abs(E - E_ref) < 1e-10 * max(1.0, abs(E_ref))
    assert abs(nP - nP_ref) < 1e-12
    dev.close()


@pytest.mark.gpu
def test_truncated_gpu_sweeps_are_variational_and_steps_match_oracle():
    """L=8, D=32, n_beta=5 (truncated): sweep energies stay above the exact spin-S value and do
    not rise between sweeps beyond the truncation allowance.  Trajectories of the GPU and the
    oracle are not compared (the Davidson vector is defined only modulo ker N_eff, so truncated
    sweeps legitimately diverge); instead theta of the first step from the same MPS must agree."""
    require_gpu()
    L, N, twoM, twoS, D, G = 8, 8, 0, 0, 32, 5
    h1, eri = inputs.hubbard_chain(L, 1.0, 4.0)
    e_ed, _, _ = fock.lowest_spin_state(L, 4, 4, h1, eri, 0)
    labels, tens = inputs.random_mps(L, N, twoM, D, 1)
    P = S.prepare(labels, tens, M.hubbard_mpo(L, 1.0, 4.0), twoS, twoM, G)
    dev = _dev(L, N, twoM, twoS, D, G, dav_tol_r=1e-8, dav_max_iter=300)
    dev.set_mps(P.mps.labels, P.mps.A, center=0)
    E, st = dev.sweep(3)
    assert all(e >= e_ed - 1e-9 for e in E)
    assert E[2] <= E[0] + 1e-6
    assert E[-1] - e_ed < 5e-3
    dev.close()


@pytest.mark.gpu
def test_checkpoint_round_trip_and_kernel_profiler():
    require_gpu()
    L, N, twoM, twoS, D, G = 6, 6, 0, 0, 16, 4
    labels, tens = inputs.random_mps(L, N, twoM, D, 4)
    dev = _dev(L, N, twoM, twoS, D, G)
    dev.set_mps(labels, tens, center=0)
    dev.canonicalize()
    lab2, ts2, c = dev.get_mps()
    assert c == 0 and len(ts2) == L
    dev2 = _dev(L, N, twoM, twoS, D, G)
    dev2.set_mps(lab2, ts2, center=c)
    assert dev.energy() == dev2.energy()
    dev.profile(True)
    dev.sweep(1)
    st = dev.kernel_stats(0)
    assert st["launches"] > 0 and st["ms"] > 0 and st["flops"] > 0
    dev.profile(False)
    dev.close()
    dev2.close()


@pytest.mark.gpu
def test_metric_cg_preconditioner_converges_to_the_same_theta():
    """precond = metric (CG steps on N_eff t = r): same theta as the oracle's solve."""
    require_gpu()
    L, N, twoM, twoS, D, G = 6, 6, 0, 0, 12, 4
    labels, tens = inputs.random_mps(L, N, twoM, D, 3)
    P = S.prepare(labels, tens, M.hubbard_mpo(L, 1.0, 4.0), twoS, twoM, G)
    dev = _dev(L, N, twoM, twoS, D, G, precond="metric", cg_steps=5, dav_tol_r=1e-9, dav_max_iter=400)
    dev.set_mps(P.mps.labels, P.mps.A, center=0)
    th, it = dev.optimize_step(0, True)
    x0 = P.two_site(0)
    mask = S.two_site_mask(P.mps.labels[0], P.mps.labels[2])
    dh, dn = P.diagonal(0)
    res = S.davidson(lambda v: P.apply(v, 0), x0, dh, dn, mask, tol_r=1e-9, max_iter=400, precond="metric",
                     apply_n=lambda v: P.apply(v, 0, which=("n",))[0], cg_steps=5)
    assert res.converged
    assert abs(th - res.theta) < 1e-9 * max(1.0, abs(res.theta))
    dev.close()


@pytest.mark.gpu
def test_olsen_correction_converges_to_the_same_theta():
    """precond = olsen (diagonal correction made N-orthogonal to x): the solve converges to the
    oracle's lowest generalised eigenvalue, the same as with the diagonal correction."""
    require_gpu()
    L, N, twoM, twoS, D, G = 6, 6, 0, 0, 12, 4
    labels, tens = inputs.random_mps(L, N, twoM, D, 3)
    P = S.prepare(labels, tens, M.hubbard_mpo(L, 1.0, 4.0), twoS, twoM, G)
    dev = _dev(L, N, twoM, twoS, D, G, precond="olsen", dav_tol_r=1e-9, dav_max_iter=400)
    dev.set_mps(P.mps.labels, P.mps.A, center=0)
    th, it = dev.optimize_step(0, True)
    x0 = P.two_site(0)
    mask = S.two_site_mask(P.mps.labels[0], P.mps.labels[2])
    dh, dn = P.diagonal(0)
    res = S.davidson(lambda v: P.apply(v, 0), x0, dh, dn, mask, tol_r=1e-9, max_iter=400)
    assert res.converged
    assert abs(th - res.theta) < 1e-9 * max(1.0, abs(res.theta))
    dev.close()


@pytest.mark.gpu
@pytest.mark.parametrize("smem_max", [0, 8])
def test_eight_site_untruncated_sweeps_reach_ed(smem_max):
    """L=8 half filling, D=256 (no truncation: the exact middle-bond rank is 256), n_beta=5:
    the sweep energy equals the lowest S=0 eigenvalue of the 4900-dimensional sector.  With
    jacobi_smem_max=8 every decimation block above 8 is diagonalised in global memory."""
    require_gpu()
    L, N, D, G = 8, 8, 256, 5
    h1, eri = inputs.hubbard_chain(L, 1.0, 4.0)
    e_ed, _, _ = fock.lowest_spin_state(L, 4, 4, h1, eri, 0)
    labels, tens = inputs.random_mps(L, N, 0, D, 1)
    dev = _dev(L, N, 0, 0, D, G, dav_tol_r=1e-8, dav_max_iter=400, jacobi_smem_max=smem_max)
    dev.set_mps(labels, tens, center=0)
    dev.canonicalize()
    E, st = dev.sweep(4)
    assert abs(E[-1] - e_ed) < 1e-10, (E, e_ed)
    assert abs(dev.expect_s2()) < 1e-9
    dev.close()
