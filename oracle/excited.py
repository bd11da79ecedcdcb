"""State-specific excited states of SP-MPS (oracle; test infrastructure only).

Sec. 2.3.2 (Eq. orthoB, Fig. spmpsex): the first excited state |Psi_1> of spin S is optimised like
the ground state, subject at every local step to <Psi_0|P|Psi_1> = 0 with |Psi_0> the (already
optimised) lower state.  With x the two-site tensor of |Psi_1>, the overlap is linear in x,
<Psi_0|P|Psi_1> = B . x, B = <Psi_0|P|d Psi_1 / d x> (the network of Fig. spmpsex (a) with x removed).
For several lower states the B vectors are orthonormalised by a QR decomposition into V, and the
local problem (Eq. geproblem) is solved in the range of Q = 1 - V V^T.

The B network: P = sum_g c_g exp(-i b_g S_y) (Eq. pmpo) acting on the ket |Psi_1>; per beta point
the left and right environments of <Psi_0| r_g ... r_g |Psi_1> (the rotated identity MPO, bra =
Psi_0, ket = Psi_1), contracted with the two-site tensor x0 = A0[k] A0[k+1] of the lower state.
"""
from __future__ import annotations

import numpy as np

from .mpo import identity_mpo, rotate_mpo
from .mps import MPS, SweepLog, decimate, davidson, two_site_mask, sweep_schedule, min_norm_representative, METRIC_SHIFT
from .quadrature import projector_quadrature


def cross_left_update(L, A_bra, A_ket, W):
    """L'[b, v, b'] = sum A_bra[a,s,b] L[a,w,a'] W[w,v,s,t] A_ket[a',t,b']."""
    T = np.einsum("awc,ctd->awtd", L, A_ket)
    T = np.einsum("awtd,wvst->avsd", T, W)
    return np.einsum("asb,avsd->bvd", A_bra, T)


def cross_right_update(R, A_bra, A_ket, W):
    """R'[a, w, a'] = sum A_bra[a,s,b] W[w,v,s,t] R[b,v,b'] A_ket[a',t,b']."""
    T = np.einsum("ctd,bvd->ctbv", A_ket, R)
    T = np.einsum("ctbv,wvst->cswb", T, W)
    return np.einsum("asb,cswb->awc", A_bra, T)


class Overlap:
    """Per-beta environments of <Psi_0| exp(-i b_g S_y) |Psi_1>: bra = a fixed lower state, ket =
    the MPS being optimised (``ket`` is shared with that MPS's Projected object)."""

    def __init__(self, lower: MPS, ket: MPS, twoS: int, twoM: int, n_beta: int):
        self.lower = lower
        self.ket = ket
        self.beta, self.c = projector_quadrature(twoS, twoM, n_beta)
        K = ket.K
        self.W = [rotate_mpo(identity_mpo(K), b) for b in self.beta]
        G = len(self.beta)
        self.L = [[None] * (K + 1) for _ in range(G)]
        self.R = [[None] * (K + 1) for _ in range(G)]
        for g in range(G):
            self.L[g][0] = np.ones((1, 1, 1))
            self.R[g][K] = np.ones((1, 1, 1))

    def update_left(self, site: int):
        for g in range(len(self.beta)):
            self.L[g][site + 1] = cross_left_update(self.L[g][site], self.lower.A[site], self.ket.A[site], self.W[g][site])

    def update_right(self, site: int):
        for g in range(len(self.beta)):
            self.R[g][site] = cross_right_update(self.R[g][site + 1], self.lower.A[site], self.ket.A[site],
                                                 self.W[g][site])

    def build(self, k: int):
        """Environments for the two-site step at (k, k+1): left up to bond k, right down to k+2."""
        for i in range(k):
            self.update_left(i)
        for i in range(self.ket.K - 1, k + 1, -1):
            self.update_right(i)

    def B(self, k: int) -> np.ndarray:
        """B[a1, t1, t2, b1] = sum_g c_g sum x0[a0,s1,s2,b0] L_g[a0,0,a1] r_g[s1,t1] r_g[s2,t2] R_g[b0,0,b1],
        on the (N, M)-allowed entries of the ket's two-site tensor (Eq. orthoB)."""
        x0 = np.einsum("asc,cjb->asjb", self.lower.A[k], self.lower.A[k + 1])
        acc = 0.0
        for g, cg in enumerate(self.c):
            r1, r2 = self.W[g][k][0, 0], self.W[g][k + 1][0, 0]
            acc = acc + cg * np.einsum("asjb,ac,st,ju,bd->ctud", x0, self.L[g][k][:, 0, :], r1, r2, self.R[g][k + 2][:, 0, :])
        mask = two_site_mask(self.ket.labels[k], self.ket.labels[k + 2])
        return np.where(mask, acc, 0.0)


def constrained_step(P, overlaps, k: int, move_right: bool, D: int, log: SweepLog, **dav):
    """One two-site step of the excited state: the B vectors of every lower state (Eq. orthoB),
    orthonormalised by QR into V, constrain Eq. geproblem to the range of Q = 1 - V V^T; then
    decimation and the environment updates of the state and of its overlaps."""
    mps = P.mps
    x0 = P.two_site(k)
    ql, qr = mps.labels[k], mps.labels[k + 2]
    mask = two_site_mask(ql, qr)
    sel = mask.reshape(-1)
    Bs = np.stack([ov.B(k).reshape(-1)[sel] for ov in overlaps], axis=1)
    V, _ = np.linalg.qr(Bs)
    dh, dn = P.diagonal(k)
    blocks = None
    if dav.get("precond") == "metric_block":
        blocks = P.metric_blocks(k)
        dav = dict(dav, metric_blocks=blocks)
    res = davidson(lambda v: P.apply(v, k), x0, dh, dn, mask,
                   apply_n=lambda v: P.apply(v, k, which=("n",))[0], constraints=V, **dav)
    x = res.x
    if blocks is not None:
        nx = P.apply(x, k, which=("n",))[0].reshape(-1)[sel]
        full = np.zeros(mask.size)
        xm = min_norm_representative(x.reshape(-1)[sel], nx, blocks, dav.get("metric_shift", METRIC_SHIFT))
        xm = xm - V @ (V.T @ xm)
        full[sel] = xm
        x = full.reshape(mask.shape)
    Al, Ar, lm, disc = decimate(x, ql, qr, D, move_right)
    mps.A[k], mps.A[k + 1] = Al, Ar
    mps.labels[k + 1] = lm
    if move_right:
        P.update_left(k)
        for ov in overlaps:
            ov.update_left(k)
        mps.center = k + 1
    else:
        P.update_right(k + 1)
        for ov in overlaps:
            ov.update_right(k + 1)
        mps.center = k
    log.theta.append(res.theta)
    log.iterations.append(res.iterations)
    log.discarded.append(disc)
    return res


def run_excited_sweeps(P, overlaps, D: int, n_sweeps: int, log: SweepLog | None = None, **dav) -> SweepLog:
    """Two-site sweeps of the excited state from an MPS with its centre on site 0, right
    environments built for P and the overlaps."""
    log = log or SweepLog()
    for _ in range(n_sweeps):
        for k, mr in sweep_schedule(P.mps.K):
            constrained_step(P, overlaps, k, mr, D, log, **dav)
        log.sweep_energy.append(log.theta[-1])
    return log
