"""Exact diagonalisation in Fock space (oracle; test infrastructure only).

Eq. FSwf / Eq. sqH: states are occupation strings over 2K spin-orbitals; the Hamiltonian is
H = sum_{pq,s} h_pq a+_ps a_qs + 1/2 sum_{pqrs,s,t} (pq|rs) a+_ps a+_rt a_st a_qs + e_core,
with chemist integrals (pq|rs) = <pr|qs>, i.e. the paper's g_{pq,sr} = <pq|sr> = (ps|qr).
Jordan-Wigner order (Sec. 2.1): spatial orbital k holds spin-orbital 2k (alpha) then 2k+1
(beta); the sign of a_p / a+_p is (-1)^(number of occupied spin-orbitals before p).
The full Fock space is also viewed as a K-fold tensor with local index 2*n_alpha + n_beta
(the basis of Eq. Sfac), which is where the site rotations of Eq. expSy act.
"""
from __future__ import annotations

from itertools import combinations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _popcount(a: np.ndarray) -> np.ndarray:
    return np.bitwise_count(a.astype(np.uint64)).astype(np.int64)


def sector_basis(K: int, Na: int, Nb: int) -> np.ndarray:
    """Sorted bitmasks (uint64) of all determinants with Na alpha and Nb beta electrons."""
    if not (0 <= Na <= K and 0 <= Nb <= K):
        return np.zeros(0, dtype=np.uint64)
    out = []
    for ca in combinations(range(K), Na):
        ma = sum(1 << (2 * k) for k in ca)
        for cb in combinations(range(K), Nb):
            out.append(ma | sum(1 << (2 * k + 1) for k in cb))
    return np.array(sorted(out), dtype=np.uint64)


def _apply_op(masks, signs, valid, p: int, create: bool):
    bit = np.uint64(1) << np.uint64(p)
    occ = (masks & bit) != 0
    ok = valid & (~occ if create else occ)
    below = masks & (bit - np.uint64(1))
    par = _popcount(below) & 1
    signs = np.where(par == 1, -signs, signs)
    masks = masks ^ bit
    return masks, signs, ok


def operator_string(basis_in: np.ndarray, basis_out: np.ndarray, ops, coef: float):
    """Sparse matrix of coef * (product of ops), ops given left to right as
    (spin_orbital, create) and applied right to left, from span(basis_in) to span(basis_out)."""
    masks = basis_in.copy()
    signs = np.ones(len(masks))
    valid = np.ones(len(masks), dtype=bool)
    for p, create in reversed(ops):
        masks, signs, valid = _apply_op(masks, signs, valid, p, create)
    cols = np.nonzero(valid)[0]
    m = masks[cols]
    rows = np.searchsorted(basis_out, m)
    rows = np.minimum(rows, len(basis_out) - 1)
    hit = basis_out[rows] == m
    cols, rows = cols[hit], rows[hit]
    return sp.csr_matrix((coef * signs[cols], (rows, cols)), shape=(len(basis_out), len(basis_in)))


def hamiltonian(K: int, Na: int, Nb: int, h1: np.ndarray, eri: np.ndarray | None, ecore: float = 0.0):
    """Sparse H of Eq. sqH on the (Na, Nb) sector."""
    basis = sector_basis(K, Na, Nb)
    n = len(basis)
    H = sp.csr_matrix((n, n))
    for p in range(K):
        for q in range(K):
            if h1[p, q] == 0.0:
                continue
            for s in (0, 1):
                H = H + operator_string(basis, basis, [(2 * p + s, True), (2 * q + s, False)], h1[p, q])
    if eri is not None:
        for p, q, r, s_ in zip(*np.nonzero(eri)):
            v = 0.5 * eri[p, q, r, s_]
            for s in (0, 1):
                for t in (0, 1):
                    ops = [(2 * p + s, True), (2 * r + t, True), (2 * s_ + t, False), (2 * q + s, False)]
                    H = H + operator_string(basis, basis, ops, v)
    if ecore:
        H = H + ecore * sp.identity(n, format="csr")
    return H.tocsr(), basis


def s_plus(K: int, Na: int, Nb: int):
    """S+ = sum_k a+_{k alpha} a_{k beta} from sector (Na, Nb) to (Na+1, Nb-1)."""
    bin_ = sector_basis(K, Na, Nb)
    bout = sector_basis(K, Na + 1, Nb - 1)
    S = sp.csr_matrix((len(bout), len(bin_)))
    if len(bout) == 0:
        return S
    for k in range(K):
        S = S + operator_string(bin_, bout, [(2 * k, True), (2 * k + 1, False)], 1.0)
    return S.tocsr()


def s_squared(K: int, Na: int, Nb: int):
    """S^2 = S- S+ + Sz (Sz + 1) on the (Na, Nb) sector."""
    sz = 0.5 * (Na - Nb)
    Sp = s_plus(K, Na, Nb)
    n = len(sector_basis(K, Na, Nb))
    return (Sp.T @ Sp + sz * (sz + 1.0) * sp.identity(n)).tocsr()


def lowest_spin_state(K, Na, Nb, h1, eri, twoS, ecore=0.0, penalty=None):
    """Lowest eigenpair of H restricted to S^2 = S(S+1) in the (Na, Nb) sector, from the
    penalised operator H + mu (S^2 - S(S+1))^2 (S^2 built from creation operators)."""
    H, basis = hamiltonian(K, Na, Nb, h1, eri, ecore)
    S2 = s_squared(K, Na, Nb)
    s = 0.5 * twoS
    n = H.shape[0]
    A = S2 - s * (s + 1) * sp.identity(n)
    if penalty is None:
        penalty = 10.0 * (1.0 + abs(spla.norm(H, 1)))
    Hp = (H + penalty * (A @ A)).tocsr()
    if n <= 400:
        w, v = np.linalg.eigh(Hp.toarray())
        e, vec = w[0], v[:, 0]
    else:
        w, v = spla.eigsh(Hp, k=1, which="SA", tol=1e-13, maxiter=100000)
        e, vec = w[0], v[:, 0]
    return e, vec, basis


# ---- tensor-product (site) view ---------------------------------------------------------

def mask_to_sites(masks: np.ndarray, K: int) -> np.ndarray:
    """Flat index of the K-site tensor (site 0 most significant, local 2*n_a + n_b)."""
    idx = np.zeros(len(masks), dtype=np.int64)
    for k in range(K):
        na = ((masks >> np.uint64(2 * k)) & np.uint64(1)).astype(np.int64)
        nb = ((masks >> np.uint64(2 * k + 1)) & np.uint64(1)).astype(np.int64)
        idx = idx * 4 + 2 * na + nb
    return idx


def embed(vec: np.ndarray, basis: np.ndarray, K: int) -> np.ndarray:
    full = np.zeros(4 ** K)
    full[mask_to_sites(basis, K)] = vec
    return full


def restrict(full: np.ndarray, basis: np.ndarray, K: int) -> np.ndarray:
    return full[mask_to_sites(basis, K)]


def apply_site_ops(full: np.ndarray, ops: list[np.ndarray]) -> np.ndarray:
    """Apply one 4x4 matrix per site to a K-site tensor."""
    K = len(ops)
    t = full.reshape((4,) * K)
    for k, o in enumerate(ops):
        t = np.moveaxis(np.tensordot(o, t, axes=([1], [k])), 0, k)
    return t.reshape(-1)


def total_sy_generator(K: int, N: int):
    """Real matrix G = -i S_y = -(S+ - S-)/2 on the fixed-N part of Fock space (all M),
    built from creation/annihilation operators; exp(beta G) = exp(-i beta S_y)."""
    blocks = []
    for na in range(0, N + 1):
        nb = N - na
        if 0 <= na <= K and 0 <= nb <= K:
            blocks.append((na, nb, sector_basis(K, na, nb)))
    basis = np.concatenate([b for (_, _, b) in blocks])
    order = np.argsort(basis)
    basis = basis[order]
    n = len(basis)
    G = sp.csr_matrix((n, n))
    for k in range(K):
        Sp = operator_string(basis, basis, [(2 * k, True), (2 * k + 1, False)], 1.0)
        G = G - 0.5 * (Sp - Sp.T)
    return G.tocsr(), basis
