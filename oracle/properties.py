"""Spin-free properties of the spin-projected state (oracle; test infrastructure only).

Eq. PropSpinFree: for an operator O that commutes with the projector,
<O> = <Psi|O P|Psi> / <Psi|P|Psi>, Psi the underlying (N, M) MPS.  Written out on the full
Fock sector for small K: Psi is contracted to a vector, P applied as the Gauss-Legendre sum of
products of site rotations (Eq. pmpo, Eq. expSy), and O built from creation / annihilation
operators by the ED code.  The operators are the ones the paper names: the fragment energies
e_p (the terms of Eq. sumH with first creation operator on spatial orbital p, both spins), the
spin-free one-particle density matrix E_pq = sum_s a+_ps a_qs, spin-spin correlations
S_X . S_Y between orbital sets, and the seniority number operator (singly occupied orbitals).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fock
from .mps import MPS, to_full_vector
from .quadrature import projector_quadrature, site_rotation


def _sector(mps: MPS, K: int, N: int, twoM: int):
    Na, Nb = (N + twoM) // 2, (N - twoM) // 2
    basis = fock.sector_basis(K, Na, Nb)
    return Na, Nb, basis, fock.mask_to_sites(basis, K)


def projected_pair(mps: MPS, K: int, N: int, twoM: int, twoS: int, n_beta: int):
    """(psi, P psi) restricted to the (N, M) sector."""
    Na, Nb, basis, idx = _sector(mps, K, N, twoM)
    full = to_full_vector(mps)
    beta, c = projector_quadrature(twoS, twoM, n_beta)
    pf = sum(cg * fock.apply_site_ops(full, [site_rotation(b)] * K) for b, cg in zip(beta, c))
    return full[idx], pf[idx], (Na, Nb, basis)


def expectation(O, psi: np.ndarray, ppsi: np.ndarray) -> float:
    """Eq. PropSpinFree with O a sector matrix."""
    return float(psi @ (O @ ppsi)) / float(psi @ ppsi)


def fragment_operator(K, Na, Nb, h1, eri, p):
    """The terms of H (Eq. sqH, chemist integrals) whose first creation operator is on spatial
    orbital p, both spins: the group sum_s H_{p s} of Eq. sumH."""
    h1m = np.zeros_like(h1)
    h1m[p, :] = h1[p, :]
    erim = None
    if eri is not None:
        erim = np.zeros_like(eri)
        erim[p] = eri[p]
    H, _ = fock.hamiltonian(K, Na, Nb, h1m, erim)
    return H


def excitation_operator(K, Na, Nb, p, q):
    """E_pq = sum_s a+_{p s} a_{q s}."""
    e = np.zeros((K, K))
    e[p, q] = 1.0
    H, _ = fock.hamiltonian(K, Na, Nb, e, None)
    return H


def spin_dot_operator(K, Na, Nb, X, Y):
    """S_X . S_Y = 1/2 (S+_X S-_Y + S-_X S+_Y) + Sz_X Sz_Y with S+_i = a+_{i a} a_{i b},
    S-_i = a+_{i b} a_{i a}, Sz_i = (n_{i a} - n_{i b}) / 2, summed over i in X and j in Y."""
    basis = fock.sector_basis(K, Na, Nb)
    n = len(basis)
    O = sp.csr_matrix((n, n))
    for i in X:
        for j in Y:
            # S+_i S-_j and S-_i S+_j as four-operator strings (each conserves the sector)
            O = O + fock.operator_string(basis, basis, [(2 * i, True), (2 * i + 1, False), (2 * j + 1, True), (2 * j, False)], 0.5)
            O = O + fock.operator_string(basis, basis, [(2 * i + 1, True), (2 * i, False), (2 * j, True), (2 * j + 1, False)], 0.5)
    # Sz_X Sz_Y is diagonal
    occ = np.array([[(int(m) >> (2 * k)) & 1 for k in range(K)] for m in basis], dtype=float).reshape(n, K)
    occb = np.array([[(int(m) >> (2 * k + 1)) & 1 for k in range(K)] for m in basis], dtype=float).reshape(n, K)
    sz = 0.5 * (occ - occb)
    d = sz[:, list(X)].sum(axis=1) * sz[:, list(Y)].sum(axis=1)
    return (O + sp.diags(d)).tocsr()


def seniority_operator(K, Na, Nb):
    """Omega = sum_k (n_{k a} + n_{k b} - 2 n_{k a} n_{k b}): the number of singly occupied orbitals."""
    basis = fock.sector_basis(K, Na, Nb)
    d = np.zeros(len(basis))
    for k in range(K):
        a = (basis >> np.uint64(2 * k)) & np.uint64(1)
        b = (basis >> np.uint64(2 * k + 1)) & np.uint64(1)
        d += (a ^ b).astype(float)
    return sp.diags(d).tocsr()
