"""The library's general MPO (spmps_mpo_from_integrals, host only) against exact
diagonalisation: Eq. sqH on the whole Fock space, any integrals (Eq. sumH does not use their
symmetry), and the bond dimensions of the complementary-operator channels."""
import numpy as np
import pytest

from oracle import fock, mpo as M
from paper_1703_04789_gb300 import inputs


def _lib_mpo(h1, eri, ecore=0.0):
    from paper_1703_04789_gb300 import mpo_from_integrals
    from tests.gpu_util import library
    library()
    return mpo_from_integrals(h1, eri, ecore)


def _dense_fock(K, h1, eri, ecore):
    Hf = np.zeros((4 ** K, 4 ** K))
    for Na in range(K + 1):
        for Nb in range(K + 1):
            H, basis = fock.hamiltonian(K, Na, Nb, h1, eri, ecore)
            idx = fock.mask_to_sites(basis, K)
            Hf[np.ix_(idx, idx)] = H.toarray()
    return Hf


@pytest.mark.parametrize("K,symmetric", [(2, False), (3, False), (3, True), (4, True), (4, False)])
def test_library_mpo_equals_ed(K, symmetric):
    if symmetric:
        h1, eri, _ = inputs.synthetic_active_space(K, 7)
    else:
        rng = np.random.default_rng(70 + K)
        h1 = rng.standard_normal((K, K))
        eri = rng.standard_normal((K, K, K, K))
    ws = _lib_mpo(h1, eri, -0.61)
    Hd = M.mpo_to_dense(ws)
    assert np.abs(Hd - _dense_fock(K, h1, eri, -0.61)).max() < 1e-12


def test_library_mpo_one_body_only_and_hubbard():
    rng = np.random.default_rng(3)
    h1 = rng.standard_normal((3, 3))
    h1 = h1 + h1.T
    assert np.abs(M.mpo_to_dense(_lib_mpo(h1, None)) - _dense_fock(3, h1, None, 0.0)).max() < 1e-12
    h1, eri = inputs.hubbard_chain(3, 1.0, 4.0)
    assert np.abs(M.mpo_to_dense(_lib_mpo(h1, eri)) - M.mpo_to_dense(M.hubbard_mpo(3, 1.0, 4.0))).max() < 1e-12


@pytest.mark.parametrize("K", [4, 6, 10])
def test_library_mpo_bond_dimensions(K):
    """With dense integrals every channel appears: at a cut with nL / nR spin-orbitals on its
    sides, 2 (start, done) + 2 nL + 2 nR (one operator on one side) + 2 m^2 - m (operator pairs
    of the smaller side, m = min(nL, nR))."""
    h1, eri, _ = inputs.synthetic_active_space(K, 1)
    ws = _lib_mpo(h1, eri)
    dims = [1] + [w.shape[1] for w in ws]
    for b in range(1, K):
        nL, nR = 2 * b, 2 * (K - b)
        m = min(nL, nR)
        assert dims[b] == 2 + 2 * nL + 2 * nR + 2 * m * m - m, (b, dims[b])
    assert dims[0] == dims[K] == 1
