"""The projected action and sweeps with a general (ab initio) Hamiltonian on the GPU.

The oracle builds H as the sum of MPOs of Eq. sumH (Eq. Wfac per term, direct sum); the
library builds its own complementary-operator MPO from the same integrals.  The two share
nothing but the integrals, the MPS and x, so agreement of y, z (element by element) and of the
sweep energies with exact diagonalisation checks the library's MPO, environments and action
together.  Integrals: the synthetic active-space recipe (h1 diag U(-3,-1), off-diagonal
N(0, 0.1), (pp|qq) U(0.3, 0.8), other entries N(0, 0.02), 8-fold symmetric).
"""
import numpy as np
import pytest

from oracle import fock, mpo as M, mps as S, quadrature as Q
from paper_1703_04789_gb300 import inputs
from tests.gpu_util import masked_random_two_site, require_gpu

RTOL = 1e-10

CASES = [
    # K, N, 2M, 2S, D, n_beta, seed
    (4, 4, 0, 0, 8, 3, 1),
    (5, 6, 2, 2, 12, 4, 2),
    (6, 9, 3, 3, 16, 4, 3),   # N_alpha = K: every state of the sector has S = M (P = 1)
    (6, 6, 0, 0, 12, 4, 4),
]


def _setup(K, N, twoM, twoS, D, G, seed):
    from paper_1703_04789_gb300 import Spmps
    h1, eri, ecore = inputs.synthetic_active_space(K, seed)
    labels, tens = inputs.random_mps(K, N, twoM, D, seed)
    P = S.prepare(labels, tens, M.ab_initio_mpo(h1, eri, ecore), twoS, twoM, G)
    dev = Spmps(K, N, twoM, twoS, G, D)
    dev.set_hamiltonian(h1, eri, ecore)
    dev.set_mps(P.mps.labels, P.mps.A, center=0)
    return P, dev, (h1, eri)


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES)
def test_ab_initio_apply_matches_oracle_every_site(case):
    require_gpu()
    K, N, twoM, twoS, D, G, seed = case
    P, dev, _ = _setup(*case)
    rng = np.random.default_rng(seed + 2000)
    P.build_left(K - 2)
    for k in range(K - 1):
        ql, qr = P.mps.labels[k], P.mps.labels[k + 2]
        lay = dev.x_layout(k)
        x = masked_random_two_site(ql, qr, rng)
        y_ref, z_ref = P.apply(x, k)
        yv, zv = dev.apply_heff_host(k, dev.pack(x, lay, ql, qr))
        y = dev.unpack(yv, lay, ql, qr)
        z = dev.unpack(zv, lay, ql, qr)
        assert np.abs(y - y_ref).max() <= RTOL * max(1.0, np.abs(y_ref).max()), k
        assert np.abs(z - z_ref).max() <= RTOL * max(1.0, np.abs(z_ref).max()), k
    E, nP = dev.energy()
    E_ref, nP_ref = P.energy(0)
    assert abs(E - E_ref) < 1e-10 and abs(nP - nP_ref) < 1e-12
    dev.close()


@pytest.mark.gpu
@pytest.mark.parametrize("K,N,twoM,twoS,D,G", [(4, 4, 0, 0, 16, 3), (4, 4, 2, 2, 16, 3), (5, 5, 1, 3, 32, 4)])
def test_ab_initio_untruncated_sweeps_reach_exact_spin_state(K, N, twoM, twoS, D, G):
    require_gpu()
    from paper_1703_04789_gb300 import Spmps
    h1, eri, ecore = inputs.synthetic_active_space(K, 11)
    Na, Nb = inputs.electron_counts(N, twoM)
    e_ed, _, _ = fock.lowest_spin_state(K, Na, Nb, h1, eri, twoS, ecore)
    labels, tens = inputs.random_mps(K, N, twoM, D, 5)
    dev = Spmps(K, N, twoM, twoS, G, D, dav_tol_r=1e-8)
    dev.set_hamiltonian(h1, eri, ecore)
    dev.set_mps(labels, tens, center=0)
    dev.canonicalize()
    E, _ = dev.sweep(4)
    assert abs(E[-1] - e_ed) < 1e-8, (E, e_ed)
    s = 0.5 * twoS
    assert abs(dev.expect_s2() - s * (s + 1)) < 1e-8
    dev.close()


@pytest.mark.gpu
def test_high_spin_sector_projector_is_identity():
    """N_alpha = K: every determinant of the sector has S = M, so <P> = 1 for any MPS and the
    projected energy is the plain expectation value <H>."""
    require_gpu()
    K, N, twoM, twoS, D, G, seed = 6, 9, 3, 3, 16, 4, 3
    P, dev, (h1, eri) = _setup(K, N, twoM, twoS, D, G, seed)
    E, nP = dev.energy()
    assert abs(nP - 1.0) < 1e-12
    # plain <H>: the same MPS with the identity in place of the projector
    full = S.to_full_vector(P.mps)
    Na, Nb = inputs.electron_counts(N, twoM)
    H, basis = fock.hamiltonian(K, Na, Nb, h1, eri)
    v = full[fock.mask_to_sites(basis, K)]
    assert abs(E - float(v @ (H @ v)) / float(v @ v)) < 1e-10
    dev.close()


@pytest.mark.gpu
def test_set_mpo_matches_set_hamiltonian():
    """The same operator handed over as MPO site tensors (spmps_set_mpo) gives the same action."""
    require_gpu()
    from paper_1703_04789_gb300 import Spmps
    K, N, twoM, twoS, D, G, seed = 5, 6, 2, 2, 12, 4, 2
    h1, eri, ecore = inputs.synthetic_active_space(K, seed)
    labels, tens = inputs.random_mps(K, N, twoM, D, seed)
    a = Spmps(K, N, twoM, twoS, G, D)
    b = Spmps(K, N, twoM, twoS, G, D)
    a.set_hamiltonian(h1, eri, ecore)
    b.set_mpo(M.ab_initio_mpo(h1, eri, ecore))
    for dev in (a, b):
        dev.set_mps(labels, tens, center=0)
        dev.canonicalize()
    k = 1
    xv = np.random.default_rng(0).standard_normal(a.x_layout(k)["n_x"])
    ya, za = a.apply_heff_host(k, xv)
    yb, zb = b.apply_heff_host(k, xv)
    assert np.abs(ya - yb).max() < 1e-10 * max(1.0, np.abs(ya).max())
    assert np.abs(za - zb).max() < 1e-12 * max(1.0, np.abs(za).max())
    a.close()
    b.close()
