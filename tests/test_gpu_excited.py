"""State-specific excited states on the GPU (Sec. 2.3.2, Eq. orthoB, Fig. spmpsex) against the oracle
and exact diagonalisation.

B_j = <Psi_j| P |d Psi / d x> is built from per-beta environments between the running state and
the lower state; <Psi_j|P|Psi> = B_j . x is compared with the oracle's network (1e-11 relative),
the constrained local problem's theta with the oracle's constrained solve (1e-9), and untruncated
constrained sweeps must reach the second-lowest spin-S eigenvalue of exact diagonalisation
(1e-8) with the projected overlap to the ground state below 1e-7.
"""
import numpy as np
import pytest

from oracle import excited as X, fock, mpo as M, mps as S, quadrature as Q
from paper_1703_04789_gb300 import inputs
from tests.gpu_util import require_gpu


def _dev(K, N, twoM, twoS, D, G, **kw):
    from paper_1703_04789_gb300 import Spmps
    d = Spmps(K, N, twoM, twoS, G, D, **kw)
    d.set_hubbard(1.0, 4.0)
    return d


@pytest.mark.gpu
@pytest.mark.parametrize("K,N,twoM,twoS,D", [(6, 6, 0, 0, 12), (7, 7, 1, 3, 16), (8, 8, 2, 2, 24)])
def test_lower_overlap_matches_oracle(K, N, twoM, twoS, D):
    require_gpu()
    G = Q.n_exact(K, N, twoM, twoS)
    l0, t0 = inputs.random_mps(K, N, twoM, D, 11)
    l1, t1 = inputs.random_mps(K, N, twoM, D, 12)
    m0 = S.MPS([q.copy() for q in l0], [t.copy() for t in t0], 0)
    m1 = S.MPS([q.copy() for q in l1], [t.copy() for t in t1], 0)
    ov = X.Overlap(m0, m1, twoS, twoM, G)
    ov.build(0)
    ref = float(np.vdot(ov.B(0), np.einsum("asc,cjb->asjb", m1.A[0], m1.A[1])))
    dev = _dev(K, N, twoM, twoS, D, G)
    dev.set_mps(l1, t1, center=0)
    dev.add_lower_state(l0, t0)
    val = dev.lower_overlap(0)
    assert abs(val - ref) <= 1e-11 * max(1.0, abs(ref)), (val, ref)
    dev.close()


@pytest.mark.gpu
def test_constrained_step_theta_matches_oracle():
    require_gpu()
    K, N, twoM, twoS, D = 8, 8, 0, 0, 24
    G = Q.n_exact(K, N, twoM, twoS)
    l0, t0 = inputs.random_mps(K, N, twoM, D, 3)
    l1, t1 = inputs.random_mps(K, N, twoM, D, 4)
    P1 = S.prepare(l1, t1, M.hubbard_mpo(K, 1.0, 4.0), twoS, twoM, G)
    m0 = S.MPS([q.copy() for q in l0], [t.copy() for t in t0], 0)
    ov = X.Overlap(m0, P1.mps, twoS, twoM, G)
    ov.build(0)
    x0 = P1.two_site(0)
    mask = S.two_site_mask(P1.mps.labels[0], P1.mps.labels[2])
    sel = mask.reshape(-1)
    V, _ = np.linalg.qr(ov.B(0).reshape(-1)[sel][:, None])
    dh, dn = P1.diagonal(0)
    res = S.davidson(lambda v: P1.apply(v, 0), x0, dh, dn, mask, tol_r=1e-9, max_iter=400, constraints=V)
    assert res.converged
    dev = _dev(K, N, twoM, twoS, D, G, dav_tol_r=1e-9, dav_max_iter=400)
    dev.set_mps(P1.mps.labels, P1.mps.A, center=0)
    dev.add_lower_state(l0, t0)
    th, it = dev.optimize_step(0, True)
    assert abs(th - res.theta) < 1e-9 * max(1.0, abs(res.theta)), (th, res.theta, it)
    dev.close()


@pytest.mark.gpu
@pytest.mark.parametrize("K,N,twoM,twoS,D", [(6, 6, 0, 0, 64), (6, 6, 2, 2, 64)])
def test_excited_state_sweeps_reach_ed(K, N, twoM, twoS, D):
    require_gpu()
    G = Q.n_exact(K, N, twoM, twoS)
    h1, eri = inputs.hubbard_chain(K, 1.0, 4.0)
    Na, Nb = inputs.electron_counts(N, twoM)
    H, _ = fock.hamiltonian(K, Na, Nb, h1, eri)
    S2 = fock.s_squared(K, Na, Nb).toarray()
    s = 0.5 * twoS
    A = S2 - s * (s + 1) * np.eye(S2.shape[0])
    w = np.linalg.eigvalsh(H.toarray() + 50.0 * A @ A)
    gs = _dev(K, N, twoM, twoS, D, G, dav_tol_r=1e-9, dav_max_iter=300)
    l0, t0 = inputs.random_mps(K, N, twoM, D, 1)
    gs.set_mps(l0, t0, center=0)
    gs.canonicalize()
    E0, _ = gs.sweep(3)
    assert abs(E0[-1] - w[0]) < 1e-8, (E0, w[:3])
    lab0, ts0, _ = gs.get_mps()
    gs.close()
    ex = _dev(K, N, twoM, twoS, D, G, dav_tol_r=1e-9, dav_max_iter=300)
    l1, t1 = inputs.random_mps(K, N, twoM, D, 7)
    ex.set_mps(l1, t1, center=0)
    ex.canonicalize()
    ex.add_lower_state(lab0, ts0)
    E1, _ = ex.sweep(3)
    assert abs(E1[-1] - w[1]) < 1e-8, (E1, w[:3])
    assert abs(ex.lower_overlap(0)) < 1e-7
    ex.close()
