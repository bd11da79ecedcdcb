"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks an oracle function against something that is not the oracle itself:
textbook values, closed forms, values the paper states, a library routine on a special
case, brute force on tiny inputs, or an invariant of the method.
"""
import os
from math import comb, sqrt

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.special import eval_legendre

from oracle import fock, mpo as M, mps as S, quadrature as Q
from paper_1703_04789_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


# ---- quadrature (Eq. pmpo, Eq. exactQuadrature) ------------------------------------------

def test_gauss_legendre_textbook_values():
    ref = _load("gauss_legendre_5.txt")
    x, w = Q.gauss_legendre(5)
    assert np.allclose(x, ref[:, 0], atol=1e-10)
    assert np.allclose(w, ref[:, 1], atol=1e-10)
    # 3-point closed form: nodes 0, +-sqrt(3/5), weights 8/9, 5/9
    x3, w3 = Q.gauss_legendre(3)
    assert np.allclose(x3, [-sqrt(0.6), 0.0, sqrt(0.6)], atol=1e-15)
    assert np.allclose(w3, [5 / 9, 8 / 9, 5 / 9], atol=1e-15)


@pytest.mark.parametrize("n", [1, 3, 5, 8, 12])
def test_gauss_legendre_exact_degree(n):
    x, w = Q.gauss_legendre(n)
    for k in range(2 * n):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.dot(w, x ** k) - exact) < 1e-13
    k = 2 * n
    assert abs(np.dot(w, x ** k) - 2.0 / (k + 1)) > 1e-9  # degree 2n is not integrated exactly


@pytest.mark.parametrize("beta", [0.0, 0.3, 1.1, 2.0, np.pi])
def test_wigner_d_closed_forms(beta):
    d = Q.wigner_small_d
    assert abs(d(1, 1, 1, beta) - np.cos(beta / 2)) < 1e-14
    assert abs(d(1, -1, -1, beta) - np.cos(beta / 2)) < 1e-14
    assert abs(d(1, 1, -1, beta) + np.sin(beta / 2)) < 1e-14
    assert abs(d(2, 0, 0, beta) - np.cos(beta)) < 1e-14
    assert abs(d(2, 2, 2, beta) - (1 + np.cos(beta)) / 2) < 1e-14
    assert abs(d(2, 2, 0, beta) + np.sin(beta) / sqrt(2)) < 1e-14
    for two_j in range(0, 12, 2):
        assert abs(d(two_j, 0, 0, beta) - eval_legendre(two_j // 2, np.cos(beta))) < 1e-12


@pytest.mark.parametrize("two_j", [1, 2, 3, 4, 7])
def test_wigner_d_orthogonal_rows(two_j):
    beta = 0.77
    ms = range(-two_j, two_j + 1, 2)
    Dm = np.array([[Q.wigner_small_d(two_j, a, b, beta) for b in ms] for a in ms])
    assert np.allclose(Dm @ Dm.T, np.eye(len(ms)), atol=1e-13)
    assert np.allclose(np.array([[Q.wigner_small_d(two_j, a, b, 0.0) for b in ms] for a in ms]), np.eye(len(ms)))


def test_exact_quadrature_rule_values():
    for K, N, twoM, twoS, ng in _load("exact_quadrature.txt").astype(int):
        assert Q.n_exact(K, N, twoM, twoS) == ng, (K, N, twoM, twoS)


@pytest.mark.parametrize("twoM", [0, 2])
def test_discrete_orthogonality_of_d(twoM):
    """With n points, sum_g (2S+1)/2 w_g d^S_MM d^S'_MM = delta_SS' whenever the product is a
    polynomial in cos(beta) of degree <= 2n-1 (both have degree <= S)."""
    n = 5
    x, w = Q.gauss_legendre(n)
    beta = np.arccos(x)
    Ss = [s for s in range(abs(twoM), 12, 2) if (s + s) // 2 <= 2 * n - 1]
    for a in Ss:
        for b in Ss:
            if (a + b) // 2 > 2 * n - 1:
                continue
            val = 0.5 * (a + 1) * sum(wg * Q.wigner_small_d(a, twoM, twoM, bg) * Q.wigner_small_d(b, twoM, twoM, bg)
                                      for wg, bg in zip(w, beta))
            assert abs(val - (1.0 if a == b else 0.0)) < 1e-12, (a, b)


# ---- rotations (Eq. expSy) ----------------------------------------------------------------

def test_site_rotation_is_exponential_of_local_sy():
    gen = -0.5 * (M.S_PLUS - M.S_MINUS)  # -i S_y, real
    for b in (0.1, 1.3, 2.9):
        assert np.allclose(Q.site_rotation(b), sla.expm(b * gen), atol=1e-14)


@pytest.mark.parametrize("K,N", [(2, 2), (3, 3), (3, 4)])
def test_product_of_site_rotations_is_many_body_rotation(K, N):
    G, basis = fock.total_sy_generator(K, N)
    beta = 0.9
    R = sla.expm(beta * G.toarray())
    idx = fock.mask_to_sites(basis, K)
    rng = np.random.default_rng(0)
    v = rng.standard_normal(len(basis))
    full = np.zeros(4 ** K)
    full[idx] = v
    out = fock.apply_site_ops(full, [Q.site_rotation(beta)] * K)
    assert np.allclose(out[idx], R @ v, atol=1e-13)
    assert np.allclose(np.delete(out, idx), 0.0, atol=1e-14)  # rotation keeps N


# ---- exact diagonalisation (Eq. sqH) -------------------------------------------------------

def test_hubbard_dimer_closed_form():
    for U in (0.0, 1.0, 4.0, 8.0):
        h1, eri = inputs.hubbard_chain(2, 1.0, U)
        e, _, _ = fock.lowest_spin_state(2, 1, 1, h1, eri, 0)
        assert abs(e - (U - sqrt(U * U + 16.0)) / 2) < 1e-12
        et, _, _ = fock.lowest_spin_state(2, 2, 0, h1, eri, 2)
        assert abs(et) < 1e-12


@pytest.mark.parametrize("L,twoS", [(8, 0), (8, 2), (24, 0), (24, 2)])
def test_free_chain_single_particle_sum(L, twoS):
    """U = 0 open chain: E = sum of occupied levels -2t cos(pi j/(L+1)); checked on ED for L=8
    and on the closed form's known values for L=24 (no ED)."""
    levels = np.sort(-2.0 * np.cos(np.pi * np.arange(1, L + 1) / (L + 1)))
    Na, Nb = (L + twoS) // 2, (L - twoS) // 2
    e_cf = levels[:Na].sum() + levels[:Nb].sum()
    known = {(8, 0): -9.5175409663, (8, 2): -8.8229482556, (24, 0): -29.8519422198, (24, 2): -29.6007801417}
    assert abs(e_cf - known[(L, twoS)]) < 1e-9
    if L <= 8:
        h1, eri = inputs.hubbard_chain(L, 1.0, 0.0)
        e, _, _ = fock.lowest_spin_state(L, Na, Nb, h1, None, twoS)
        assert abs(e - e_cf) < 1e-9


def test_random_one_body_ground_state_is_orbital_sum():
    """General (non-nearest-neighbour) h1 exercises every Jordan-Wigner string."""
    K = 5
    rng = np.random.default_rng(7)
    h1 = rng.standard_normal((K, K))
    h1 = h1 + h1.T
    eps = np.linalg.eigvalsh(h1)
    for Na, Nb in ((2, 2), (3, 1), (3, 2)):
        H, _ = fock.hamiltonian(K, Na, Nb, h1, None)
        e = np.linalg.eigvalsh(H.toarray())[0]
        assert abs(e - eps[:Na].sum() - eps[:Nb].sum()) < 1e-10


def test_two_body_slater_condon_diagonal():
    """<D|H|D> = sum_i h_ii + 1/2 sum_ij [(ii|jj) - delta_{s_i s_j} (ij|ji)] for every
    determinant D (fixes the sign of exchange and the 1/2)."""
    K = 4
    h1, eri, _ = inputs.synthetic_active_space(K, 11)
    H, basis = fock.hamiltonian(K, 2, 1, h1, eri)
    Hd = H.diagonal()
    for j, m in enumerate(basis):
        occ = [(p // 2, p % 2) for p in range(2 * K) if (int(m) >> p) & 1]
        e = sum(h1[k, k] for k, _ in occ)
        for (k, s) in occ:
            for (l, t) in occ:
                e += 0.5 * eri[k, k, l, l]
                if s == t:
                    e -= 0.5 * eri[k, l, l, k]
        assert abs(Hd[j] - e) < 1e-12


def test_hamiltonian_is_spin_free():
    K = 4
    h1, eri, _ = inputs.synthetic_active_space(K, 3)
    H, _ = fock.hamiltonian(K, 2, 2, h1, eri)
    S2 = fock.s_squared(K, 2, 2)
    assert abs(H - H.T).max() < 1e-13
    assert abs(H @ S2 - S2 @ H).max() < 1e-12


def test_atomic_limit():
    """t = 0: the lowest S=0 energy at half filling is 0 (no double occupancy), with two
    extra electrons it is 2U."""
    h1, eri = inputs.hubbard_chain(4, 0.0, 3.0)
    e, _, _ = fock.lowest_spin_state(4, 2, 2, h1, eri, 0)
    assert abs(e) < 1e-12
    e, _, _ = fock.lowest_spin_state(4, 3, 3, h1, eri, 0)
    assert abs(e - 6.0) < 1e-12


# ---- MPOs (Eq. Wfac merged to spatial sites, Eq. Sfac) -------------------------------------

@pytest.mark.parametrize("L", [2, 3, 4])
def test_hubbard_mpo_equals_ed(L):
    h1, eri = inputs.hubbard_chain(L, 1.3, 2.7)
    Hd = M.mpo_to_dense(M.hubbard_mpo(L, 1.3, 2.7))
    for Na in range(L + 1):
        for Nb in range(L + 1):
            H, basis = fock.hamiltonian(L, Na, Nb, h1, eri)
            idx = fock.mask_to_sites(basis, L)
            assert np.allclose(Hd[np.ix_(idx, idx)], H.toarray(), atol=1e-13)


@pytest.mark.parametrize("K", [2, 3, 4])
def test_s2_mpo_equals_ed(K):
    S2d = M.mpo_to_dense(M.s2_mpo(K))
    for Na in range(K + 1):
        for Nb in range(K + 1):
            basis = fock.sector_basis(K, Na, Nb)
            idx = fock.mask_to_sites(basis, K)
            assert np.allclose(S2d[np.ix_(idx, idx)], fock.s_squared(K, Na, Nb).toarray(), atol=1e-13)


def _dense_fock_hamiltonian(K, h1, eri, ecore):
    """The full 4^K matrix of Eq. sqH assembled sector by sector from the ED code."""
    Hf = np.zeros((4 ** K, 4 ** K))
    for Na in range(K + 1):
        for Nb in range(K + 1):
            H, basis = fock.hamiltonian(K, Na, Nb, h1, eri, ecore)
            idx = fock.mask_to_sites(basis, K)
            Hf[np.ix_(idx, idx)] = H.toarray()
    return Hf


@pytest.mark.parametrize("K,symmetric", [(2, False), (3, False), (3, True), (4, True)])
def test_ab_initio_mpo_equals_ed(K, symmetric):
    """Eq. sumH / Eq. Wfac merged to spatial sites reproduces the Fock-space H of Eq. sqH on the
    whole 4^K space (every (Na, Nb) block and zero between blocks); the construction does not
    use the symmetry of the integrals, so a general eri is checked too."""
    if symmetric:
        h1, eri, _ = inputs.synthetic_active_space(K, 3)
    else:
        rng = np.random.default_rng(40 + K)
        h1 = rng.standard_normal((K, K))
        eri = rng.standard_normal((K, K, K, K))
    Hd = M.mpo_to_dense(M.ab_initio_mpo(h1, eri, 0.37))
    assert np.abs(Hd - _dense_fock_hamiltonian(K, h1, eri, 0.37)).max() < 1e-12


def test_ab_initio_mpo_reduces_to_hubbard():
    """Hubbard integrals (h1 = -t on the chain, (pp|pp) = U) through the general construction give
    the same operator as the hand-built Hubbard MPO."""
    h1, eri = inputs.hubbard_chain(3, 1.1, 3.3)
    a = M.mpo_to_dense(M.ab_initio_mpo(h1, eri))
    b = M.mpo_to_dense(M.hubbard_mpo(3, 1.1, 3.3))
    assert np.abs(a - b).max() < 1e-12


# ---- the projector (Eq. PSMM, Eq. pmpo) ----------------------------------------------------

def _projector_matrix(K, N, twoM, twoS, n_beta):
    Na, Nb = inputs.electron_counts(N, twoM)
    basis = fock.sector_basis(K, Na, Nb)
    idx = fock.mask_to_sites(basis, K)
    beta, c = Q.projector_quadrature(twoS, twoM, n_beta)
    P = np.zeros((len(basis), len(basis)))
    for j in range(len(basis)):
        full = np.zeros(4 ** K)
        full[idx[j]] = 1.0
        acc = sum(cg * fock.apply_site_ops(full, [Q.site_rotation(b)] * K) for b, cg in zip(beta, c))
        P[:, j] = acc[idx]
    return P, basis


@pytest.mark.parametrize("K,N,twoM,twoS", [(4, 4, 0, 0), (4, 4, 0, 2), (5, 5, 1, 1), (5, 5, 1, 3), (4, 4, 2, 2)])
def test_projector_idempotent_symmetric_and_counts_multiplets(K, N, twoM, twoS):
    ng = Q.n_exact(K, N, twoM, twoS)
    P, basis = _projector_matrix(K, N, twoM, twoS, ng)
    assert np.allclose(P, P.T, atol=1e-13)
    assert np.allclose(P @ P, P, atol=1e-12)
    Na, Nb = inputs.electron_counts(N, twoM)
    Ms = (N + twoS) // 2
    dimS = comb(K, Ms) * comb(K, N - Ms)
    dimS1 = comb(K, Ms + 1) * comb(K, N - Ms - 1) if N - Ms - 1 >= 0 else 0
    assert abs(np.trace(P) - (dimS - dimS1)) < 1e-10
    S2 = fock.s_squared(K, Na, Nb).toarray()
    s = 0.5 * twoS
    assert np.allclose(S2 @ P, s * (s + 1) * P, atol=1e-11)


def test_projector_with_too_few_points_is_not_idempotent():
    K, N, twoM, twoS = 4, 4, 0, 0
    ng = Q.n_exact(K, N, twoM, twoS)
    P, _ = _projector_matrix(K, N, twoM, twoS, ng - 1)
    assert np.abs(P @ P - P).max() > 1e-3


def test_singlet_count_for_eight_site_half_filling():
    # 4900 states with Sz = 0, 3136 with Sz = 1: 1764 singlets
    assert comb(8, 4) ** 2 - comb(8, 5) * comb(8, 3) == 1764


# ---- the projected action against brute force (Eq. geproblem, Fig. spmpsOpt) ---------------

def _embedding(mps, k):
    """Columns: full 4^K vectors of the two-site basis |a> |s1> |s2> |b> at (k, k+1),
    built from the MPS tensors alone."""
    K = mps.K
    left = np.ones((1, 1))
    for i in range(k):
        left = np.einsum("Xa,asb->Xsb", left, mps.A[i]).reshape(-1, mps.A[i].shape[2])
    right = np.ones((1, 1))
    for i in range(K - 1, k + 1, -1):
        right = np.einsum("asb,bY->asY", mps.A[i], right).reshape(mps.A[i].shape[0], -1)
    Dl, Dr = left.shape[1], right.shape[0]
    cols = []
    for a in range(Dl):
        for s1 in range(4):
            for s2 in range(4):
                for b in range(Dr):
                    e1 = np.zeros(4); e1[s1] = 1
                    e2 = np.zeros(4); e2[s2] = 1
                    cols.append(np.kron(np.kron(np.kron(left[:, a], e1), e2), right[b]))
    return np.array(cols).T


@pytest.mark.parametrize("K,N,twoM,twoS,D,seed", [(4, 4, 0, 0, 8, 1), (5, 5, 1, 1, 6, 2), (4, 4, 0, 2, 8, 3), (5, 4, 0, 0, 7, 4)])
def test_projected_apply_matches_brute_force(K, N, twoM, twoS, D, seed):
    U, t = 3.0, 1.0
    h1, eri = inputs.hubbard_chain(K, t, U)
    labels, tens = inputs.random_mps(K, N, twoM, D, seed)
    ng = Q.n_exact(K, N, twoM, twoS)
    P = S.prepare(labels, tens, M.hubbard_mpo(K, t, U), twoS, twoM, ng)
    # move the centre to sites (k, k+1) by left-canonical steps through the oracle itself,
    # then compare against brute force built from the MPS tensors only
    Na, Nb = inputs.electron_counts(N, twoM)
    H, basis = fock.hamiltonian(K, Na, Nb, h1, eri)
    idx = fock.mask_to_sites(basis, K)
    beta, c = Q.projector_quadrature(twoS, twoM, ng)
    rng = np.random.default_rng(seed + 100)
    for k in range(K - 1):
        V = _embedding(P.mps, k)
        ql, qr = P.mps.labels[k], P.mps.labels[k + 2]
        mask = S.two_site_mask(ql, qr)
        x = np.where(mask, rng.standard_normal(mask.shape), 0.0)
        y, z = P.apply(x, k)
        full = V @ x.reshape(-1)
        proj = sum(cg * fock.apply_site_ops(full, [Q.site_rotation(b)] * K) for b, cg in zip(beta, c))
        sec = proj[idx]
        hy = np.zeros(4 ** K); hy[idx] = H @ sec
        nz = np.zeros(4 ** K); nz[idx] = sec
        y_bf = (V.T @ hy).reshape(x.shape) * mask
        z_bf = (V.T @ nz).reshape(x.shape) * mask
        assert np.abs(y - y_bf).max() < 1e-12 * max(1.0, np.abs(y_bf).max())
        assert np.abs(z - z_bf).max() < 1e-12 * max(1.0, np.abs(z_bf).max())
        if k < K - 2:
            S.two_site_step(P, k, True, D, S.SweepLog(), max_iter=3)


def test_heff_neff_symmetric_and_metric_in_unit_interval():
    K, N, twoM, twoS, D = 5, 5, 1, 1, 8
    labels, tens = inputs.random_mps(K, N, twoM, D, 5)
    P = S.prepare(labels, tens, M.hubbard_mpo(K, 1.0, 4.0), twoS, twoM, Q.n_exact(K, N, twoM, twoS))
    k = 0
    mask = S.two_site_mask(P.mps.labels[k], P.mps.labels[k + 2])
    sel = np.nonzero(mask.reshape(-1))[0]
    Hm = np.zeros((len(sel), len(sel)))
    Nm = np.zeros_like(Hm)
    for j, p in enumerate(sel):
        e = np.zeros(mask.size); e[p] = 1.0
        y, z = P.apply(e.reshape(mask.shape), k)
        Hm[:, j] = y.reshape(-1)[sel]
        Nm[:, j] = z.reshape(-1)[sel]
    assert np.allclose(Hm, Hm.T, atol=1e-12)
    assert np.allclose(Nm, Nm.T, atol=1e-13)
    mu = np.linalg.eigvalsh(Nm)
    assert mu.min() > -1e-12 and mu.max() < 1 + 1e-12
    dh, dn = P.diagonal(k)
    assert np.allclose(dh.reshape(-1)[sel], np.diag(Hm), atol=1e-13)
    assert np.allclose(dn.reshape(-1)[sel], np.diag(Nm), atol=1e-13)


# ---- energies and sweeps -------------------------------------------------------------------

def _functional_ed(mps, h1, eri, K, N, twoM, twoS, ng):
    Na, Nb = inputs.electron_counts(N, twoM)
    H, basis = fock.hamiltonian(K, Na, Nb, h1, eri)
    psi = S.to_full_vector(mps)
    beta, c = Q.projector_quadrature(twoS, twoM, ng)
    pp = sum(cg * fock.apply_site_ops(psi, [Q.site_rotation(b)] * K) for b, cg in zip(beta, c))
    idx = fock.mask_to_sites(basis, K)
    return float(psi[idx] @ (H @ pp[idx]) / (psi[idx] @ pp[idx])), float(psi[idx] @ pp[idx])


@pytest.mark.parametrize("K,N,twoM,twoS,D,seed", [(4, 4, 0, 0, 8, 1), (5, 5, 1, 3, 8, 2)])
def test_energy_functional_matches_ed(K, N, twoM, twoS, D, seed):
    h1, eri = inputs.hubbard_chain(K, 1.0, 4.0)
    ng = Q.n_exact(K, N, twoM, twoS)
    labels, tens = inputs.random_mps(K, N, twoM, D, seed)
    P = S.prepare(labels, tens, M.hubbard_mpo(K, 1.0, 4.0), twoS, twoM, ng)
    E, nP = P.energy(0)
    E_ed, nP_ed = _functional_ed(P.mps, h1, eri, K, N, twoM, twoS, ng)
    assert abs(E - E_ed) < 1e-12
    assert abs(nP - nP_ed) < 1e-13
    assert 0.0 < nP <= 1.0 + 1e-12


@pytest.mark.parametrize("K,N,twoM,twoS,D", [(4, 4, 0, 0, 16), (4, 4, 2, 2, 16), (4, 4, 0, 2, 16), (6, 6, 0, 0, 64)])
def test_untruncated_sweeps_reach_exact_spin_state(K, N, twoM, twoS, D):
    """D at the exact Schmidt rank: sweeps reach the lowest spin-S ED eigenvalue, obtained
    independently of the projector (S^2 penalty built from creation operators)."""
    h1, eri = inputs.hubbard_chain(K, 1.0, 4.0)
    Na, Nb = inputs.electron_counts(N, twoM)
    e_ed, _, _ = fock.lowest_spin_state(K, Na, Nb, h1, eri, twoS)
    labels, tens = inputs.random_mps(K, N, twoM, D, 1)
    P = S.prepare(labels, tens, M.hubbard_mpo(K, 1.0, 4.0), twoS, twoM, Q.n_exact(K, N, twoM, twoS))
    log = S.run_sweeps(P, D, 3, tol_r=1e-9)
    assert abs(log.sweep_energy[-1] - e_ed) < 1e-10
    # <S^2> of the projected state, through the same engine with the S^2 MPO of Eq. Sfac
    P2 = S.Projected(P.mps, M.s2_mpo(K), twoS, twoM, Q.n_exact(K, N, twoM, twoS))
    P2.build_right(2)
    s2, _ = P2.energy(0)
    s = 0.5 * twoS
    assert abs(s2 - s * (s + 1)) < 1e-10


def test_truncated_sweeps_are_variational():
    K, N, twoM, twoS, D = 6, 6, 0, 0, 12
    h1, eri = inputs.hubbard_chain(K, 1.0, 4.0)
    e_ed, _, _ = fock.lowest_spin_state(K, 3, 3, h1, eri, twoS)
    labels, tens = inputs.random_mps(K, N, twoM, D, 3)
    P = S.prepare(labels, tens, M.hubbard_mpo(K, 1.0, 4.0), twoS, twoM, Q.n_exact(K, N, twoM, twoS))
    log = S.run_sweeps(P, D, 2)
    assert all(th >= e_ed - 1e-10 for th in log.theta)
    E, _ = P.energy(0)
    E_ed_fn, _ = _functional_ed(P.mps, h1, eri, K, N, twoM, twoS, Q.n_exact(K, N, twoM, twoS))
    assert abs(E - E_ed_fn) < 1e-10 and E >= e_ed - 1e-10


def test_spin_flip_leaves_singlet_functional_unchanged():
    """alpha <-> beta on every site (with |ab> -> -|ab>) commutes with a spin-free H and with
    the S=0, M=0 projector, so the functional is unchanged."""
    K, N, D = 4, 4, 8
    labels, tens = inputs.random_mps(K, N, 0, D, 9)
    flip = np.zeros((4, 4)); flip[0, 0] = 1; flip[1, 2] = 1; flip[2, 1] = 1; flip[3, 3] = -1
    ng = Q.n_exact(K, N, 0, 0)
    mpo = M.hubbard_mpo(K, 1.0, 4.0)
    P = S.prepare(labels, tens, mpo, 0, 0, ng)
    E1, _ = P.energy(0)
    flipped = [np.einsum("ts,asb->atb", flip, A) for A in P.mps.A]
    fl_labels = [np.stack([l[:, 0], -l[:, 1]], axis=1) for l in P.mps.labels]
    # re-sort the bond indices so labels stay sorted by (n, 2m)
    perms = [np.lexsort((l[:, 1], l[:, 0])) for l in fl_labels]
    fl_labels = [l[p] for l, p in zip(fl_labels, perms)]
    flipped = [A[np.ix_(perms[i], range(4), perms[i + 1])] for i, A in enumerate(flipped)]
    P2 = S.prepare(fl_labels, flipped, mpo, 0, 0, ng)
    E2, _ = P2.energy(0)
    assert abs(E1 - E2) < 1e-12


# ---- decimation and Davidson ---------------------------------------------------------------

def test_untruncated_decimation_reconstructs_and_is_canonical():
    K, N, D = 5, 5, 64
    labels, tens = inputs.random_mps(K, N, 1, 6, 4)
    P = S.prepare(labels, tens, M.hubbard_mpo(K, 1.0, 4.0), 1, 1, 2)
    k = 1
    ql, qr = P.mps.labels[k], P.mps.labels[k + 2]
    rng = np.random.default_rng(0)
    x = np.where(S.two_site_mask(ql, qr), rng.standard_normal((ql.shape[0], 4, 4, qr.shape[0])), 0.0)
    for move_right in (True, False):
        Al, Ar, lm, disc = S.decimate(x, ql, qr, D, move_right)
        rec = np.einsum("asc,cjb->asjb", Al, Ar)
        assert np.allclose(rec, x / np.linalg.norm(x), atol=1e-13)
        assert disc < 1e-24
        if move_right:
            Lm = Al.reshape(-1, Al.shape[2])
            assert np.allclose(Lm.T @ Lm, np.eye(Lm.shape[1]), atol=1e-13)
        else:
            Rm = Ar.reshape(Ar.shape[0], -1)
            assert np.allclose(Rm @ Rm.T, np.eye(Rm.shape[0]), atol=1e-13)
        assert np.all(np.diff(lm[:, 0] * 1000 + lm[:, 1]) >= 0)


def test_ordered_truncation_tie_rule():
    vals = [0.5, 0.3, 0.3 + 1e-13, 0.3, 0.1, 1e-9]
    tags = [(2, 0, 0), (3, 1, 0), (3, -1, 0), (2, 0, 1), (1, 1, 0), (0, 0, 0)]
    keep = S.ordered_truncation(vals, tags, 3)
    # 0.5 first; then the tie cluster {0.3 x 3} ordered by (n, 2m, index): (2,0,1), (3,-1,0), (3,1,0)
    assert keep == [0, 3, 2]
    assert S.ordered_truncation(vals, tags, 10) == [0, 3, 2, 1, 4]  # 1e-9 < 1e-7 dropped


@pytest.mark.parametrize("K,N,twoM,twoS,D,k", [(5, 5, 1, 1, 8, 1), (6, 6, 0, 0, 12, 2), (6, 6, 2, 2, 10, 3)])
def test_metric_blocks_are_the_exact_diagonal_blocks_of_n_eff(K, N, twoM, twoS, D, k):
    """N_eff, assembled column by column from the oracle's N network, vanishes between entries of
    different (n(a), n(s1), n(s2)) and equals metric_blocks inside each block."""
    labels, tens = inputs.random_mps(K, N, twoM, D, 7)
    P = S.prepare(labels, tens, M.hubbard_mpo(K, 1.0, 4.0), twoS, twoM, Q.n_exact(K, N, twoM, twoS))
    P.build_left(k)
    mask = S.two_site_mask(P.mps.labels[k], P.mps.labels[k + 2])
    sel = np.nonzero(mask.reshape(-1))[0]
    Nm = np.zeros((len(sel), len(sel)))
    for j, p in enumerate(sel):
        e = np.zeros(mask.size); e[p] = 1.0
        Nm[:, j] = P.apply(e.reshape(mask.shape), k, which=("n",))[0].reshape(-1)[sel]
    blocks = P.metric_blocks(k)
    covered = np.zeros_like(Nm, dtype=bool)
    assert sorted(np.concatenate([pos for pos, _ in blocks]).tolist()) == list(range(len(sel)))
    for pos, blk in blocks:
        assert np.abs(Nm[np.ix_(pos, pos)] - blk).max() < 1e-14
        covered[np.ix_(pos, pos)] = True
    assert np.abs(Nm[~covered]).max() == 0.0
    assert len(blocks) > 1


def test_min_norm_representative_keeps_the_projected_state():
    """x' = (N + shift)^-1 N x: N x' = N x up to the shift, x' has no component in ker N and
    no larger norm than x (checked against a dense eigendecomposition of N)."""
    K, N, twoM, twoS, D, k = 6, 6, 0, 0, 16, 2
    labels, tens = inputs.random_mps(K, N, twoM, D, 3)
    P = S.prepare(labels, tens, M.hubbard_mpo(K, 1.0, 4.0), twoS, twoM, Q.n_exact(K, N, twoM, twoS))
    P.build_left(k)
    mask = S.two_site_mask(P.mps.labels[k], P.mps.labels[k + 2])
    sel = np.nonzero(mask.reshape(-1))[0]
    blocks = P.metric_blocks(k)
    Nm = np.zeros((len(sel), len(sel)))
    for pos, blk in blocks:
        Nm[np.ix_(pos, pos)] = blk
    nu, V = np.linalg.eigh(Nm)
    assert (nu < 1e-12).sum() > 0  # the two-site space of this bond has a null space
    rng = np.random.default_rng(0)
    x = rng.standard_normal(len(sel))
    xp = S.min_norm_representative(x, Nm @ x, blocks, 1e-7)
    assert np.abs(Nm @ xp - Nm @ x).max() < 1e-6 * np.abs(Nm @ x).max()
    assert np.abs(V[:, nu < 1e-12].T @ xp).max() < 1e-8 * np.linalg.norm(x)
    assert np.linalg.norm(xp) <= np.linalg.norm(x)


@pytest.mark.parametrize("precond", ["diag", "metric", "metric_block"])
def test_davidson_matches_library_generalised_eigensolver(precond):
    """Special case that a library routine solves: random symmetric H, positive-definite N."""
    n = 60
    rng = np.random.default_rng(1)
    A = rng.standard_normal((n, n)); H = A + A.T + np.diag(np.arange(n, dtype=float))
    B = rng.standard_normal((n, n)); Nm = B @ B.T / n + np.eye(n)
    shape = (n,)
    ex = sla.eigh(H, Nm, eigvals_only=True)[0]
    res = S.davidson(lambda v: (H @ v, Nm @ v), rng.standard_normal(n), np.diag(H), np.diag(Nm),
                     np.ones(shape, bool), tol_r=1e-9, precond=precond, apply_n=lambda v: Nm @ v,
                     metric_blocks=[(np.arange(n), Nm)])
    assert res.converged
    assert abs(res.theta - ex) < 1e-10
    assert abs(res.x @ Nm @ res.x - 1.0) < 1e-10


# ---- learned preconditioner (oracle MLP) ---------------------------------------------------

def test_mlp_gradients_match_finite_differences():
    from oracle import mlp
    p = mlp.init_params(3)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((16, mlp.N_FEATURES))
    t = rng.standard_normal(16)
    loss, g = mlp.loss_and_grads(p, X, t)
    for key, idx in (("W1", (1, 5)), ("b1", (7,)), ("W2", (3, 11)), ("b2", (2,)), ("w3", (9,)), ("b3", (0,))):
        h = 1e-6
        q = {k: v.copy() for k, v in p.items()}
        q[key][idx] += h
        lp, _ = mlp.loss_and_grads(q, X, t)
        q[key][idx] -= 2 * h
        lm, _ = mlp.loss_and_grads(q, X, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[key][idx]) < 1e-6 * max(1.0, abs(fd)), key


def test_mlp_features_reduce_to_diagonal_preconditioner_direction():
    from oracle import mlp
    rng = np.random.default_rng(5)
    n = 50
    r, dh, dn = rng.standard_normal(n), rng.uniform(1, 2, n), rng.uniform(0.1, 0.5, n)
    f = mlp.features(r, dh, dn, -0.3)
    d = -r / (dh + 0.3 * dn)
    assert np.allclose(f[:, 1], np.sqrt(n) * d / np.linalg.norm(d))
    assert abs(np.linalg.norm(f[:, 0]) - np.sqrt(n)) < 1e-12


def test_mlp_features_metric_and_shifted_diagonal_columns():
    """Columns 2 and 3 on hand-computed values: the N_eff diagonal as given, and
    tanh((dh - theta dn) / (1 + |theta|)) with the unclamped shifted diagonal (the clamp applies only
    to the correction of column 1): theta = -2 gives scale 3."""
    from oracle import mlp
    r = np.array([1.0, -1.0, 0.5])
    dh = np.array([1.0, 0.0, -0.5])
    dn = np.array([0.25, 0.5, 0.0])
    f = mlp.features(r, dh, dn, -2.0)
    assert np.array_equal(f[:, 2], dn)
    shifted = np.array([1.0 + 0.5, 0.0 + 1.0, -0.5])  # dh - theta dn
    assert np.allclose(f[:, 3], np.tanh(shifted / 3.0), rtol=0, atol=1e-15)
    # a shifted diagonal of zero (dh = theta dn) maps to 0
    g = mlp.features(np.ones(2), np.array([0.6, -0.6]), np.array([0.3, -0.3]), 2.0)
    assert g[0, 3] == 0.0 and g[1, 3] == 0.0


def test_adam_matches_closed_form_first_step():
    from oracle import mlp
    p = {"a": np.array([1.0, -2.0])}
    g = {"a": np.array([0.5, -4.0])}
    st = {}
    mlp.adam_step(p, g, st, lr=0.1)
    # the first bias-corrected Adam step is lr * sign(g) (up to eps)
    assert np.allclose(p["a"], [1.0 - 0.1, -2.0 + 0.1], atol=1e-7)


def test_bf16_rounding_matches_known_values():
    from oracle import mlp
    # 1 + 2^-8 is exactly half-way between bf16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    assert mlp.to_bf16(np.float32(1.0 + 2.0 ** -8)) == 1.0
    assert mlp.to_bf16(np.float32(1.0 + 3 * 2.0 ** -8)) == 1.0 + 2.0 ** -6  # half-way, rounds to even (up)
    assert mlp.to_bf16(np.float32(1.0 + 2.0 ** -7)) == 1.0 + 2.0 ** -7      # representable
    assert mlp.to_bf16(np.float32(-3.0)) == -3.0


# ---- spin-free properties (Eq. PropSpinFree) ------------------------------------------------

def _prop_state(K, N, twoM, twoS, D, seed):
    from oracle import properties as PR
    h1, eri, _ = inputs.synthetic_active_space(K, seed)
    labels, tens = inputs.random_mps(K, N, twoM, D, seed)
    ng = Q.n_exact(K, N, twoM, twoS)
    P = S.prepare(labels, tens, M.ab_initio_mpo(h1, eri), twoS, twoM, ng)
    psi, ppsi, (Na, Nb, basis) = PR.projected_pair(P.mps, K, N, twoM, twoS, ng)
    return P, h1, eri, psi, ppsi, Na, Nb


@pytest.mark.parametrize("K,N,twoM,twoS", [(4, 4, 0, 0), (4, 5, 1, 3)])
def test_fragment_energies_sum_to_the_energy(K, N, twoM, twoS):
    """Eq. sumH grouped by spatial orbital: sum_p e_p is the projected energy, which the MPO
    environment code computes independently."""
    from oracle import properties as PR
    P, h1, eri, psi, ppsi, Na, Nb = _prop_state(K, N, twoM, twoS, 8, 3)
    e = [PR.expectation(PR.fragment_operator(K, Na, Nb, h1, eri, p), psi, ppsi) for p in range(K)]
    E, _ = P.energy(0)
    assert abs(sum(e) - E) < 1e-11


def test_rdm1_trace_symmetry_and_spin_sum_rule():
    """tr(gamma) = N, gamma symmetric with eigenvalues in [0, 2]; sum over all i, j of
    <S_i . S_j> = S(S+1) for the projected state."""
    from oracle import properties as PR
    K, N, twoM, twoS = 4, 4, 0, 2
    P, h1, eri, psi, ppsi, Na, Nb = _prop_state(K, N, twoM, twoS, 8, 4)
    g = np.array([[PR.expectation(PR.excitation_operator(K, Na, Nb, p, q), psi, ppsi) for q in range(K)]
                  for p in range(K)])
    assert abs(np.trace(g) - N) < 1e-12
    assert np.abs(g - g.T).max() < 1e-12
    w = np.linalg.eigvalsh(g)
    assert w.min() > -1e-12 and w.max() < 2.0 + 1e-12
    s2 = PR.expectation(PR.spin_dot_operator(K, Na, Nb, range(K), range(K)), psi, ppsi)
    assert abs(s2 - 0.5 * twoS * (0.5 * twoS + 1)) < 1e-11


def test_seniority_closed_forms():
    """The N_alpha = K sector has exactly K - N_beta = 2M singly occupied orbitals in every
    determinant; a closed-shell determinant has none."""
    from oracle import properties as PR
    K, N, twoM = 5, 8, 2
    P, h1, eri, psi, ppsi, Na, Nb = _prop_state(K, N, twoM, twoM, 6, 5)
    assert abs(PR.expectation(PR.seniority_operator(K, Na, Nb), psi, ppsi) - twoM) < 1e-12
    basis = fock.sector_basis(3, 1, 1)
    v = np.zeros(len(basis))
    v[int(np.nonzero(basis == np.uint64(0b11))[0][0])] = 1.0
    assert abs(PR.expectation(PR.seniority_operator(3, 1, 1), v, v)) < 1e-15


# ---- approximate M-sector screening (Sec. 2.3.1, closing paragraph) -------------------------

def test_screen_environment_drops_exactly_the_small_label_blocks():
    """Hand-built environment, one channel, two labels per side: (1,-1) with one index and (1,1)
    with two.  Sub-block norms 2, 0.05, 1e-3 and 10; tau = 0.01 cuts below 0.1."""
    q = np.array([[1, -1], [1, 1], [1, 1]])
    E = np.zeros((3, 1, 3))
    E[0, 0, 0] = 1e-3                      # ((1,-1), (1,-1))
    E[0, 0, 1:] = [0.03, 0.04]             # ((1,-1), (1,1)): norm 0.05
    E[1:, 0, 0] = [1.2, 1.6]               # ((1,1), (1,-1)): norm 2
    E[1:, 0, 1:] = [[6.0, 0.0], [0.0, 8.0]]  # ((1,1), (1,1)): norm 10
    out = S.screen_environment(E, q, q, 0.01)
    expect = E.copy()
    expect[0, 0, 0] = 0.0
    expect[0, 0, 1:] = 0.0
    assert np.array_equal(out, expect)
    assert np.array_equal(S.screen_environment(E, q, q, 1e-5), E)  # nothing below 1e-4


def test_screened_action_reduces_to_the_action_and_error_shrinks_with_tau():
    K, N, D, G, k = 8, 8, 32, 5, 3
    labels, tens = inputs.random_mps(K, N, 0, D, 1)
    P = S.prepare(labels, tens, M.hubbard_mpo(K, 1.0, 4.0), 0, 0, G)
    P.build_left(k)
    ql, qr = P.mps.labels[k], P.mps.labels[k + 2]
    x = np.where(S.two_site_mask(ql, qr), np.random.default_rng(0).standard_normal((ql.shape[0], 4, 4, qr.shape[0])), 0.0)
    y0, z0 = P.apply(x, k)
    y, z = P.apply(x, k, screen=1e-14)  # only sub-blocks at the rounding level are dropped
    assert np.abs(y - y0).max() <= 1e-13 * np.abs(y0).max() and np.abs(z - z0).max() <= 1e-13 * np.abs(z0).max()
    errs = []
    for tau in (1e-5, 1e-3, 1e-1):
        y, z = P.apply(x, k, screen=tau)
        errs.append(np.abs(y - y0).max() / np.abs(y0).max())
    assert 0.0 < errs[0] < errs[1] < errs[2]


# ---- state-specific excited states (Sec. 2.3.2, Eq. orthoB) -----------------------------------

def _projected_overlap_fock(mps0, mps1, K, twoS, twoM, ng):
    beta, c = Q.projector_quadrature(twoS, twoM, ng)
    p0, p1 = S.to_full_vector(mps0), S.to_full_vector(mps1)
    pp = sum(cg * fock.apply_site_ops(p1, [Q.site_rotation(b)] * K) for b, cg in zip(beta, c))
    return float(p0 @ pp)


@pytest.mark.parametrize("K,N,twoM,twoS,D,k", [(5, 5, 1, 1, 8, 1), (6, 6, 0, 0, 12, 2), (6, 6, 0, 2, 10, 0)])
def test_b_vector_gives_the_projected_overlap(K, N, twoM, twoS, D, k):
    """B . x = <Psi_0| P |Psi_1> (Eq. orthoB), against the overlap of the full Fock vectors with the
    many-body projector applied, for two unrelated random MPS (no canonical form needed)."""
    from oracle import excited as X
    ng = Q.n_exact(K, N, twoM, twoS)
    l0, t0 = inputs.random_mps(K, N, twoM, D, 11)
    l1, t1 = inputs.random_mps(K, N, twoM, D, 12)
    m0 = S.MPS([q.copy() for q in l0], [t.copy() for t in t0], 0)
    m1 = S.MPS([q.copy() for q in l1], [t.copy() for t in t1], 0)
    ov = X.Overlap(m0, m1, twoS, twoM, ng)
    ov.build(k)
    x1 = np.einsum("asc,cjb->asjb", m1.A[k], m1.A[k + 1])
    val = float(np.vdot(ov.B(k), x1))
    ref = _projected_overlap_fock(m0, m1, K, twoS, twoM, ng)
    assert abs(val - ref) < 1e-12 * max(1.0, abs(ref)), (val, ref)
    assert abs(ref) > 1e-6  # the two states do overlap, so the check is not vacuous


def test_excited_sweeps_reach_the_second_spin_state():
    """K=6 Hubbard chain at half filling, S=0, D=64 (untruncated): after the ground state, the
    constrained sweeps reach the second-lowest singlet of exact diagonalisation, orthogonal to
    the ground state in the projected metric."""
    from oracle import excited as X
    K, N, twoM, twoS, D = 6, 6, 0, 0, 64
    ng = Q.n_exact(K, N, twoM, twoS)
    h1, eri = inputs.hubbard_chain(K, 1.0, 4.0)
    Na, Nb = inputs.electron_counts(N, twoM)
    H, _ = fock.hamiltonian(K, Na, Nb, h1, eri)
    S2 = fock.s_squared(K, Na, Nb).toarray()
    w = np.linalg.eigvalsh(H.toarray() + 50.0 * S2 @ S2)
    l0, t0 = inputs.random_mps(K, N, twoM, D, 1)
    P0 = S.prepare(l0, t0, M.hubbard_mpo(K, 1.0, 4.0), twoS, twoM, ng)
    S.run_sweeps(P0, D, 3, tol_r=1e-9, max_iter=300)
    l1, t1 = inputs.random_mps(K, N, twoM, D, 7)
    P1 = S.prepare(l1, t1, M.hubbard_mpo(K, 1.0, 4.0), twoS, twoM, ng)
    ov = X.Overlap(P0.mps, P1.mps, twoS, twoM, ng)
    ov.build(0)
    log = X.run_excited_sweeps(P1, [ov], D, 3, tol_r=1e-9, max_iter=300)
    assert abs(log.sweep_energy[-1] - w[1]) < 1e-9, (log.sweep_energy, w[:3])
    assert abs(_projected_overlap_fock(P0.mps, P1.mps, K, twoS, twoM, ng)) < 1e-9
