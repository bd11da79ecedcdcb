"""Spin-free properties of the projected state on the GPU (Eq. PropSpinFree) against the oracle,
which evaluates the same expectation values on the full Fock sector."""
import numpy as np
import pytest

from oracle import mpo as M, mps as S, properties as PR, quadrature as Q
from paper_1703_04789_gb300 import inputs
from tests.gpu_util import require_gpu


def _state(K, N, twoM, twoS, D, seed, ab_initio=True):
    from paper_1703_04789_gb300 import Spmps
    if ab_initio:
        h1, eri, ecore = inputs.synthetic_active_space(K, seed)
    else:
        h1, eri = inputs.hubbard_chain(K, 1.0, 4.0)
        ecore = 0.0
    ng = Q.n_exact(K, N, twoM, twoS)
    labels, tens = inputs.random_mps(K, N, twoM, D, seed)
    P = S.prepare(labels, tens, M.ab_initio_mpo(h1, eri, ecore) if ab_initio else M.hubbard_mpo(K, 1.0, 4.0),
                  twoS, twoM, ng)
    dev = Spmps(K, N, twoM, twoS, ng, D)
    if ab_initio:
        dev.set_hamiltonian(h1, eri, ecore)
    else:
        dev.set_hubbard(1.0, 4.0)
    dev.set_mps(P.mps.labels, P.mps.A, center=0)
    psi, ppsi, (Na, Nb, _) = PR.projected_pair(P.mps, K, N, twoM, twoS, ng)
    return dev, P, h1, eri, psi, ppsi, Na, Nb


@pytest.mark.gpu
@pytest.mark.parametrize("K,N,twoM,twoS,ab", [(4, 4, 0, 0, True), (5, 5, 1, 3, True), (5, 6, 0, 2, False)])
def test_properties_match_oracle(K, N, twoM, twoS, ab):
    require_gpu()
    dev, P, h1, eri, psi, ppsi, Na, Nb = _state(K, N, twoM, twoS, 8, 2, ab)
    e = dev.fragment_energies()
    e_ref = [PR.expectation(PR.fragment_operator(K, Na, Nb, h1, eri, p), psi, ppsi) for p in range(K)]
    assert np.abs(e - np.array(e_ref)).max() < 1e-10
    E, _ = dev.energy()
    assert abs(e.sum() - E) < 1e-10
    g = dev.rdm1()
    g_ref = np.array([[PR.expectation(PR.excitation_operator(K, Na, Nb, p, q), psi, ppsi) for q in range(K)]
                      for p in range(K)])
    assert np.abs(g - g_ref).max() < 1e-10
    X, Y = [0, 1], [K - 2, K - 1]
    c = dev.spin_correlation(X, Y)
    assert abs(c - PR.expectation(PR.spin_dot_operator(K, Na, Nb, X, Y), psi, ppsi)) < 1e-10
    allk = list(range(K))
    s = 0.5 * twoS
    assert abs(dev.spin_correlation(allk, allk) - s * (s + 1)) < 1e-10
    assert abs(dev.seniority() - PR.expectation(PR.seniority_operator(K, Na, Nb), psi, ppsi)) < 1e-10
    # the Hamiltonian and its environments are untouched
    assert abs(dev.energy()[0] - E) < 1e-12
    dev.close()


@pytest.mark.gpu
def test_expect_mpo_with_the_s2_mpo_is_s_s_plus_one():
    require_gpu()
    K, N, twoM, twoS = 5, 5, 1, 3
    dev, *_ = _state(K, N, twoM, twoS, 8, 3, True)
    s = 0.5 * twoS
    assert abs(dev.expect_mpo(M.s2_mpo(K)) - s * (s + 1)) < 1e-10
    dev.close()
