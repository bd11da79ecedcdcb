"""Local operators and MPOs on spatial-orbital sites (oracle; test infrastructure only).

Eq. JWtrans gives the 2x2 Jordan-Wigner matrices of one spin-orbital; a spatial site merges
the alpha spin-orbital (first in JW order) with the beta one (Sec. 2.1, last paragraph), so
a+_alpha = a+ (x) I and a+_beta = I~ (x) a+ with I~ = sigma_z.  The local basis index is
2*n_alpha + n_beta = {0, b, a, ab}, the order of Eq. Sfac.

An MPO site tensor is stored as W[wl, wr, s, s'] (s = bra/output index, s' = ket/input);
bond 0 and bond K have dimension 1.
"""
from __future__ import annotations

import numpy as np

from .quadrature import site_rotation

# Eq. JWtrans (one spin-orbital, basis {|0>, |1>})
I2 = np.eye(2)
SZ = np.diag([1.0, -1.0])            # I~ = sigma_z
CDAG2 = np.array([[0.0, 0.0], [1.0, 0.0]])  # a+ = sigma_-
C2 = CDAG2.T                          # a  = sigma_+

I4 = np.eye(4)
CDAG_A = np.kron(CDAG2, I2)
CDAG_B = np.kron(SZ, CDAG2)
C_A = CDAG_A.T
C_B = CDAG_B.T
PAR = np.kron(SZ, SZ)                 # (-1)^(n_a + n_b): the JW string of a whole site
N_A = CDAG_A @ C_A
N_B = CDAG_B @ C_B

# Eq. Sfac local matrices, written as in the paper
S_PLUS = np.zeros((4, 4)); S_PLUS[2, 1] = 1.0
S_MINUS = S_PLUS.T.copy()
S_Z = np.diag([0.0, -0.5, 0.5, 0.0])
S_SQ = np.diag([0.0, 0.75, 0.75, 0.0])


def _boundaries(W: np.ndarray, K: int, first_row: int, last_col: int) -> list[np.ndarray]:
    sites = []
    for k in range(K):
        w = W[k] if isinstance(W, list) else W
        if k == 0:
            w = w[first_row:first_row + 1]
        if k == K - 1:
            w = w[:, last_col:last_col + 1]
        sites.append(np.ascontiguousarray(w))
    return sites


def hubbard_mpo(L: int, t: float, U: float) -> list[np.ndarray]:
    """Open-chain Hubbard H = -t sum_{i,s} (a+_{i s} a_{i+1 s} + h.c.) + U sum_i n_ia n_ib.
    Channels: 0 = nothing placed yet, 1..4 = one hopping operator placed on the left
    (a+_a P, a+_b P, P a_a, P a_b with P the site parity), 5 = complete."""
    W = np.zeros((6, 6, 4, 4))
    W[0, 0] = I4
    W[5, 5] = I4
    W[0, 5] = U * (N_A @ N_B)
    # a+_{i s} a_{i+1 s} = (a+_s P)_i (x) (a_s)_{i+1}
    W[0, 1] = CDAG_A @ PAR
    W[0, 2] = CDAG_B @ PAR
    W[1, 5] = -t * C_A
    W[2, 5] = -t * C_B
    # a+_{i+1 s} a_{i s} = (P a_s)_i (x) (a+_s)_{i+1}
    W[0, 3] = PAR @ C_A
    W[0, 4] = PAR @ C_B
    W[3, 5] = -t * CDAG_A
    W[4, 5] = -t * CDAG_B
    return _boundaries(W, L, 0, 5)


def s2_mpo(K: int) -> list[np.ndarray]:
    """Eq. Sfac: S^2 as an MPO of bond dimension 5; the left boundary picks the S^2 row
    and the right boundary the identity column."""
    W = np.zeros((5, 5, 4, 4))
    W[0, 0] = I4
    W[0, 1] = S_MINUS
    W[0, 2] = S_PLUS
    W[0, 3] = 2.0 * S_Z
    W[0, 4] = S_SQ
    W[1, 1] = I4
    W[1, 4] = S_PLUS
    W[2, 2] = I4
    W[2, 4] = S_MINUS
    W[3, 3] = I4
    W[3, 4] = S_Z
    W[4, 4] = I4
    return _boundaries(W, K, 0, 4)


def identity_mpo(K: int) -> list[np.ndarray]:
    return [I4.reshape(1, 1, 4, 4).copy() for _ in range(K)]


def rotate_mpo(mpo: list[np.ndarray], beta: float) -> list[np.ndarray]:
    """Eq. pmpo / Fig. spmpsOpt: H exp(-i beta S_y) as one MPO, the site rotation of
    Eq. expSy multiplied onto the ket (input) leg of every site tensor."""
    r = site_rotation(beta)
    return [np.einsum("abst,tu->absu", w, r) for w in mpo]


def mpo_to_dense(mpo: list[np.ndarray]) -> np.ndarray:
    """Contract an MPO to the dense 4^K x 4^K matrix (site 0 most significant)."""
    cur = mpo[0][0]  # (wr, 4, 4)
    cur = np.transpose(cur, (0, 1, 2))
    for w in mpo[1:]:
        # cur[w, S, S'] , w[w, v, s, s'] -> new[v, (S s), (S' s')]
        new = np.einsum("wAB,wvst->vAsBt", cur, w)
        d = new.shape
        cur = new.reshape(d[0], d[1] * d[2], d[3] * d[4])
    return cur[0]


# ---- ab initio Hamiltonian as a sum of MPOs (Eq. sumH, Eq. VkK-QkK, Eq. Wfac) ----------------

SM = CDAG2                 # a+ on one spin-orbital (sigma_-)
SP = C2                    # a  (sigma_+)
NUM2 = CDAG2 @ C2          # n
SM_T = SM @ SZ             # a+~ = sigma_- sigma_z
SP_T = SP @ SZ             # a~  = sigma_+ sigma_z
NUM2_T = NUM2 @ SZ         # n~  = sigma_- sigma_+ sigma_z


def spin_orbital_integrals(h1: np.ndarray, eri: np.ndarray | None):
    """Spatial h_pq and chemist (pq|rs) to spin-orbitals 2k (alpha), 2k+1 (beta)."""
    K = h1.shape[0]
    n = 2 * K
    hs = np.zeros((n, n))
    gs = np.zeros((n, n, n, n))
    for s in (0, 1):
        hs[s::2, s::2] = h1
        if eri is not None:
            for t in (0, 1):
                gs[s::2, s::2, t::2, t::2] = eri
    return hs, gs


def v_operator_mpo(h: np.ndarray, V: np.ndarray) -> list[np.ndarray]:
    """Eq. Wfac on n spin-orbital sites (local dimension 2): the MPO of
    V = sum_q h_q a_q + sum_{q, r<s} V[q, r, s] a+_q a_r a_s (entries with r >= s are ignored).

    Channels of the bond left of site b (0-based), in this order: V (the part still to be
    placed), a+_j and a_j for j >= b, Q_l and P_l for l < b (Eq. PkK, Eq. QkK), I.  The site
    tensor maps the channels of bond b (rows) to those of bond b+1 (columns) following the
    recursions Eq. VkK, Eq. PkK and Eq. QkK."""
    n = h.shape[0]
    Vu = np.triu(np.ones((n, n)), 1)[None, :, :] * V  # V[q, r, s] only for r < s
    nch = 2 * n + 2

    def ch(b):
        # channel index map of bond b
        m = {"V": 0}
        i = 1
        for j in range(b, n):
            m[("cd", j)] = i; i += 1
        for j in range(b, n):
            m[("c", j)] = i; i += 1
        for l in range(b):
            m[("Q", l)] = i; i += 1
        for l in range(b):
            m[("P", l)] = i; i += 1
        m["I"] = i
        assert i + 1 == nch
        return m

    sites = []
    for b in range(n):
        L, R = ch(b), ch(b + 1)
        W = np.zeros((nch, nch, 2, 2))
        # row V (Eq. VkK)
        W[L["V"], R["V"]] = SZ
        for r in range(b + 1, n):
            W[L["V"], R[("c", r)]] = Vu[b, b, r] * NUM2_T
        W[L["V"], R[("Q", b)]] = -SP
        W[L["V"], R[("P", b)]] = SM
        W[L["V"], R["I"]] = h[b] * SP
        # rows a+_j, a_j
        W[L[("cd", b)], R["I"]] = SM
        W[L[("c", b)], R["I"]] = SP
        for j in range(b + 1, n):
            W[L[("cd", j)], R[("cd", j)]] = SZ
            W[L[("c", j)], R[("c", j)]] = SZ
        # rows Q_l (Eq. QkK) and P_l (Eq. PkK)
        for l in range(b):
            for r in range(b + 1, n):
                W[L[("Q", l)], R[("cd", r)]] = -Vu[r, l, b] * SP_T
                W[L[("Q", l)], R[("c", r)]] = Vu[b, l, r] * SM_T
                W[L[("P", l)], R[("c", r)]] = Vu[l, b, r] * SP_T
            W[L[("Q", l)], R[("Q", l)]] = I2
            W[L[("Q", l)], R["I"]] = Vu[b, l, b] * NUM2
            W[L[("P", l)], R[("P", l)]] = I2
        W[L["I"], R["I"]] = I2
        sites.append(W)
    sites[0] = sites[0][0:1]
    sites[-1] = sites[-1][:, nch - 1:nch]
    return sites


def _times_site_ops(ops: list[np.ndarray], mpo: list[np.ndarray]) -> list[np.ndarray]:
    """(product of one-site operators) x MPO: the operator acts after the MPO (on the bra side)."""
    return [np.einsum("su,abut->abst", o, w) for o, w in zip(ops, mpo)]


def _direct_sum(terms: list[list[np.ndarray]]) -> list[np.ndarray]:
    """One MPO for the sum of MPOs with bond dimension 1 at both ends."""
    n = len(terms[0])
    out = []
    for k in range(n):
        dl = [t[k].shape[0] for t in terms]
        dr = [t[k].shape[1] for t in terms]
        d = terms[0][k].shape[2]
        if k == 0:
            W = np.concatenate([t[0] for t in terms], axis=1)
        elif k == n - 1:
            W = np.concatenate([t[k] for t in terms], axis=0)
        else:
            W = np.zeros((sum(dl), sum(dr), d, d))
            o1 = o2 = 0
            for t, a, b in zip(terms, dl, dr):
                W[o1:o1 + a, o2:o2 + b] = t[k]
                o1 += a
                o2 += b
        out.append(W)
    return out


def merge_spin_orbital_pairs(mpo2: list[np.ndarray]) -> list[np.ndarray]:
    """Sec. 2.1, last paragraph: contract the MPO tensors of spin-orbitals 2k (alpha) and 2k+1
    (beta) into one spatial site with local index 2*n_alpha + n_beta."""
    out = []
    for k in range(len(mpo2) // 2):
        a, b = mpo2[2 * k], mpo2[2 * k + 1]
        W = np.einsum("lmst,mruv->lrsutv", a, b)
        out.append(W.reshape(a.shape[0], b.shape[1], 4, 4))
    return out


def ab_initio_mpo(h1: np.ndarray, eri: np.ndarray | None, ecore: float = 0.0) -> list[np.ndarray]:
    """Eq. sqH as the sum of MPOs of Eq. sumH: H = sum_p a+_p V_p with
    V_p = sum_q h_pq a_q + sum_{q, r<s} gA_pqrs a+_q a_r a_s and
    gA_pqrs = (g_{pq,sr} - g_{pq,rs}) / 2, g_{pq,sr} = <pq|sr> = (ps|qr) (chemist integrals in
    spin-orbitals).  Each term a+_p V_p is the MPO of Eq. Wfac times the one-site operators of
    a+_p (sigma_z on the spin-orbitals before p, sigma_- on p); the terms (and e_core times the
    identity) are summed as one MPO by direct sum and merged to spatial sites."""
    K = h1.shape[0]
    hs, gs = spin_orbital_integrals(h1, eri)
    n = 2 * K
    terms = []
    for p in range(n):
        gA = 0.5 * (np.einsum("sqr->qrs", gs[p]) - np.einsum("rqs->qrs", gs[p]))
        vp = v_operator_mpo(hs[p], gA)
        ops = [SZ] * p + [SM] + [I2] * (n - p - 1)
        terms.append(_times_site_ops(ops, vp))
    if ecore != 0.0:
        terms.append([ecore * I2.reshape(1, 1, 2, 2)] + [I2.reshape(1, 1, 2, 2).copy() for _ in range(n - 1)])
    return merge_spin_orbital_pairs(_direct_sum(terms))
