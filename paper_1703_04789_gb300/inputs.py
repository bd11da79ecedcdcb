"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module draws random numbers and lays out block structure; it contains none of the
SP-MPS arithmetic (no projector, no environments, no contraction, no canonicalisation).

Conventions (both sides read them from here):

* spatial orbitals are the MPS sites, k = 0 .. K-1 (Sec. 2.1, last paragraph);
* the local basis of a site is {|0>, |b>, |a>, |ab>} with index 2*n_alpha + n_beta
  (Eq. Sfac's basis); its particle number and twice-Sz are ``LOCAL_N`` and ``LOCAL_2M``;
* bond i (i = 0 .. K) carries the quantum numbers (n, 2m) accumulated over sites 0 .. i-1,
  so bond 0 is (0, 0) and bond K is (N, 2M); the indices of a bond are sorted by (n, 2m)
  and the indices sharing a label are contiguous.
"""
from __future__ import annotations

from math import comb

import numpy as np

LOCAL_N = (0, 1, 1, 2)
LOCAL_2M = (0, -1, 1, 0)


def electron_counts(N: int, twoM: int) -> tuple[int, int]:
    if (N + twoM) % 2:
        raise ValueError("N + 2M must be even")
    return (N + twoM) // 2, (N - twoM) // 2


def bond_sectors(K: int, N: int, twoM: int, i: int) -> list[tuple[int, int, int, int]]:
    """Labels (n, 2m) on bond i that are reachable from the left and completable on the
    right, with the number of left and right Fock states of that label."""
    Na, Nb = electron_counts(N, twoM)
    out = []
    for na in range(i + 1):
        for nb in range(i + 1):
            ra, rb = Na - na, Nb - nb
            if 0 <= ra <= K - i and 0 <= rb <= K - i:
                left = comb(i, na) * comb(i, nb)
                right = comb(K - i, ra) * comb(K - i, rb)
                out.append((na + nb, na - nb, left, right))
    out.sort(key=lambda t: (t[0], t[1]))
    return out


def _largest_remainder(weights: list[int], total: int) -> list[int]:
    s = sum(weights)
    if s <= total:
        return list(weights)
    shares = [total * w / s for w in weights]
    base = [int(np.floor(x)) for x in shares]
    rem = total - sum(base)
    order = sorted(range(len(weights)), key=lambda j: (-(shares[j] - base[j]), j))
    for j in order[:rem]:
        base[j] += 1
    return base


def mps_structure(K: int, N: int, twoM: int, D: int) -> list[list[tuple[int, int, int]]]:
    """Bond structure of the random initial MPS: for each bond 0..K a list of
    (n, 2m, dim), sorted by (n, 2m), dims split in proportion to min(left, right)
    Fock-sector sizes with largest-remainder rounding so the total is <= D.
    Labels that cannot be connected to a live label on both neighbouring bonds are
    removed (repeated until stable)."""
    bonds = []
    for i in range(K + 1):
        sec = bond_sectors(K, N, twoM, i)
        dims = _largest_remainder([min(l, r) for (_, _, l, r) in sec], D)
        bonds.append({(n, m): d for (n, m, _, _), d in zip(sec, dims) if d > 0})
    changed = True
    while changed:
        changed = False
        for i in range(1, K + 1):
            for q in list(bonds[i]):
                ok = any((q[0] - LOCAL_N[s], q[1] - LOCAL_2M[s]) in bonds[i - 1] for s in range(4))
                if not ok:
                    del bonds[i][q]
                    changed = True
        for i in range(K - 1, -1, -1):
            for q in list(bonds[i]):
                ok = any((q[0] + LOCAL_N[s], q[1] + LOCAL_2M[s]) in bonds[i + 1] for s in range(4))
                if not ok:
                    del bonds[i][q]
                    changed = True
    return [[(n, m, d) for (n, m), d in sorted(b.items())] for b in bonds]


def bond_index_labels(bond: list[tuple[int, int, int]]) -> np.ndarray:
    """Per-index (n, 2m) array of shape (D, 2) for one bond."""
    rows = [(n, m) for (n, m, d) in bond for _ in range(d)]
    return np.array(rows, dtype=np.int64).reshape(-1, 2)


def site_mask(ql: np.ndarray, qr: np.ndarray) -> np.ndarray:
    """Boolean (Dl, 4, Dr) mask of the entries allowed by (N, M) conservation."""
    dq = np.stack([np.array(LOCAL_N), np.array(LOCAL_2M)], axis=1)  # (4, 2)
    tgt = ql[:, None, :] + dq[None, :, :]  # (Dl, 4, 2)
    return np.all(tgt[:, :, None, :] == qr[None, None, :, :], axis=-1)


def random_mps(K: int, N: int, twoM: int, D: int, seed: int):
    """Raw (not canonical, not normalised) random MPS: i.i.d. N(0,1) entries on the
    allowed positions, drawn from numpy PCG64 ``default_rng(seed)`` as one
    (Dl, 4, Dr) array per site in site order.  Returns (labels, tensors) with
    labels[i] the (D_i, 2) per-index label array of bond i."""
    struct = mps_structure(K, N, twoM, D)
    labels = [bond_index_labels(b) for b in struct]
    rng = np.random.default_rng(seed)
    tensors = []
    for i in range(K):
        ql, qr = labels[i], labels[i + 1]
        draw = rng.standard_normal((ql.shape[0], 4, qr.shape[0]))
        tensors.append(np.where(site_mask(ql, qr), draw, 0.0))
    return labels, tensors


def hubbard_chain(L: int, t: float = 1.0, U: float = 4.0):
    """Open 1D Hubbard chain as one- and two-electron integrals: h[i, i+1] = h[i+1, i] = -t,
    chemist (ii|ii) = U.  Returns (h1 (L, L), eri (L, L, L, L))."""
    h1 = np.zeros((L, L))
    for i in range(L - 1):
        h1[i, i + 1] = h1[i + 1, i] = -t
    eri = np.zeros((L, L, L, L))
    for i in range(L):
        eri[i, i, i, i] = U
    return h1, eri


def _symmetrize_eri(e: np.ndarray) -> np.ndarray:
    perms = [(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2),
             (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0), (3, 2, 1, 0)]
    return sum(np.transpose(e, p) for p in perms) / 8.0


def synthetic_active_space(K: int, seed: int):
    """Random real integrals with 8-fold symmetry: h1 diag ~ U(-3,-1), off-diag ~ N(0,0.1)
    symmetric; (pp|qq) ~ U(0.3,0.8) symmetric in (p,q), every other independent entry
    ~ N(0, 0.02); ecore = 0."""
    rng = np.random.default_rng(seed)
    h1 = rng.normal(0.0, 0.1, (K, K))
    h1 = np.triu(h1, 1)
    h1 = h1 + h1.T
    h1[np.diag_indices(K)] = rng.uniform(-3.0, -1.0, K)
    eri = _symmetrize_eri(rng.normal(0.0, 0.02, (K, K, K, K)))
    coul = rng.uniform(0.3, 0.8, (K, K))
    coul = np.triu(coul) + np.triu(coul, 1).T
    for p in range(K):
        for q in range(K):
            eri[p, p, q, q] = coul[p, q]
    return h1, eri, 0.0
