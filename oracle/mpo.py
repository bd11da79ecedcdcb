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
