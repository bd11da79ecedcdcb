"""SP-MPS optimisation, plain float64 (oracle; test infrastructure only).

Tensors are dense NumPy arrays whose entries outside the (N, M) symmetry pattern are zero;
every bond carries a per-index (n, 2m) label array (left-accumulated quantum numbers).

What is computed, with the passage it follows:

* Eq. efunctional: E = <Psi| H P |Psi> / <Psi| P |Psi>, P = sum_g c_g exp(-i b_g S_y)
  (Eq. pmpo), evaluated as a sum over g of networks with the rotated MPO of each g.
* Fig. spmpsOpt / Eq. geproblem: for the two-site tensor x at sites (k, k+1) of a
  mixed-canonical MPS, H_eff x = sum_g c_g [L_g W^g_k W^g_k+1 R_g] x and
  N_eff x = sum_g c_g [LN_g r_g r_g RN_g] x, where the ket (input) side is rotated and the
  bra (output) keeps good (N, M): outputs are kept only on the (N, M)-allowed entries
  (Sec. 2.3.1, last paragraph: the rotated trial vector keeps N only and the result is
  projected back to (N, M)).
* Eq. geproblem solved by a generalised Davidson iteration (details are not in the paper:
  Euclidean-orthonormal basis, canonical orthogonalisation of the projected metric,
  lowest Ritz value, diagonal preconditioner or the inverse of the metric's symmetry blocks).
* The metric N_eff of Fig. spmpsOpt (c) is the network of the rotated identity MPO, so it is a
  sum over g of c_g L^N_g (x) r_g (x) r_g (x) R^N_g.  Each factor conserves the particle number
  of its own part (left block, site k, site k+1, right block), hence N_eff is exactly
  block-diagonal in (n of the left index, n(s1), n(s2)); ``metric_blocks`` assembles those
  blocks densely from the factors.
* Sec. 2.3.1: decimation by SVD in the usual canonical gauge; two-site sweeps.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .mpo import rotate_mpo, identity_mpo
from .quadrature import projector_quadrature

LOCAL_Q = np.array([[0, 0], [1, -1], [1, 1], [2, 0]], dtype=np.int64)  # (n, 2m) of {0,b,a,ab}
METRIC_SHIFT = 1e-7  # shift of the metric blocks in precond="metric_block" (|N_eff| <= 1)
METRIC_FLOOR = 1e-14  # Ritz problem: n-eigenvalues below this are numerically zero


def site_mask(ql, qr):
    tgt = ql[:, None, :] + LOCAL_Q[None, :, :]
    return np.all(tgt[:, :, None, :] == qr[None, None, :, :], axis=-1)


def two_site_mask(ql, qr):
    """Entries (a, s1, s2, b) of a two-site tensor with q(a) + q(s1) + q(s2) = q(b)."""
    tgt = ql[:, None, None, :] + LOCAL_Q[None, :, None, :] + LOCAL_Q[None, None, :, :]
    return np.all(tgt[:, :, :, None, :] == qr[None, None, None, :, :], axis=-1)


@dataclass
class MPS:
    labels: list          # K+1 arrays (D_i, 2)
    A: list               # K arrays (D_i, 4, D_{i+1})
    center: int = 0

    @property
    def K(self):
        return len(self.A)


def right_canonicalize(labels, tensors) -> MPS:
    """Bring sites 1..K-1 to right-canonical form by an LQ factorisation per left label
    (QR of the transpose of the allowed columns), push the factor into the left neighbour,
    and normalise site 0.  Bond dimensions of a label shrink to the rank bound
    min(rows, allowed columns) when needed."""
    labels = [l.copy() for l in labels]
    A = [t.copy() for t in tensors]
    K = len(A)
    for i in range(K - 1, 0, -1):
        ql, qr = labels[i], labels[i + 1]
        mask = site_mask(ql, qr)
        new_rows_labels = []
        new_blocks = []   # (label, Q^T rows (k, 4*Dr))
        left_factors = []  # (old row indices, R^T (r, k))
        for q in np.unique(ql, axis=0):
            rows = np.nonzero(np.all(ql == q, axis=1))[0]
            cmask = mask[rows[0]].reshape(-1)
            cols = np.nonzero(cmask)[0]
            M = A[i][rows].reshape(len(rows), -1)[:, cols]
            if len(cols) == 0:
                continue
            Q, R = np.linalg.qr(M.T, mode="reduced")  # M^T = Q R  ->  M = R^T Q^T
            k = Q.shape[1]
            blk = np.zeros((k, 4 * qr.shape[0]))
            blk[:, cols] = Q.T
            new_blocks.append(blk)
            new_rows_labels.extend([tuple(q)] * k)
            left_factors.append((rows, R.T))
        nl = np.array(new_rows_labels, dtype=np.int64).reshape(-1, 2)
        Ai = np.concatenate(new_blocks, axis=0).reshape(len(nl), 4, qr.shape[0])
        prev = A[i - 1]
        newprev = np.zeros((prev.shape[0], 4, len(nl)))
        off = 0
        for rows, Rt in left_factors:
            k = Rt.shape[1]
            newprev[:, :, off:off + k] = np.einsum("asr,rk->ask", prev[:, :, rows], Rt)
            off += k
        A[i] = Ai
        A[i - 1] = newprev
        labels[i] = nl
    A[0] = A[0] / np.linalg.norm(A[0])
    return MPS(labels, A, 0)


# ---- environments ------------------------------------------------------------------------

def left_env_update(L, A, W):
    """L'[b, v, b'] = sum A[a,s,b] L[a,w,a'] W[w,v,s,t] A[a',t,b'] (bra = A, ket = A)."""
    T = np.einsum("awc,ctd->awtd", L, A)
    T = np.einsum("awtd,wvst->avsd", T, W)
    return np.einsum("asb,avsd->bvd", A, T)


def right_env_update(R, A, W):
    """R'[a, w, a'] = sum A[a,s,b] W[w,v,s,t] R[b,v,b'] A[a',t,b']."""
    T = np.einsum("ctd,bvd->ctbv", A, R)
    T = np.einsum("ctbv,wvst->cswb", T, W)
    return np.einsum("asb,cswb->awc", A, T)


def screen_environment(E, q_bra, q_ket, tau):
    """Approximate M-sector screening (Sec. 2.3.1, closing paragraph: for a state near the target
    spin the rotation introduces few states in the other M sectors).  For every channel w of the
    environment E[a, w, a'] (bra index a, ket index a'), the sub-blocks (label(a), label(a')) whose
    Frobenius norm is below tau times the largest sub-block norm of that channel are set to zero."""
    out = E.copy()
    lb = [np.nonzero(np.all(q_bra == q, axis=1))[0] for q in np.unique(q_bra, axis=0)]
    lk = [np.nonzero(np.all(q_ket == q, axis=1))[0] for q in np.unique(q_ket, axis=0)]
    for w in range(E.shape[1]):
        norms = np.array([[np.linalg.norm(E[np.ix_(a, [w], c)]) for c in lk] for a in lb])
        cut = tau * norms.max() if norms.size else 0.0
        for i, a in enumerate(lb):
            for j, c in enumerate(lk):
                if norms[i, j] < cut:
                    out[np.ix_(a, [w], c)] = 0.0
    return out


class Projected:
    """Per-beta environments of H exp(-i b_g S_y) and of exp(-i b_g S_y) for one MPS."""

    def __init__(self, mps: MPS, mpo: list, twoS: int, twoM: int, n_beta: int):
        self.mps = mps
        self.mpo = mpo
        self.beta, self.c = projector_quadrature(twoS, twoM, n_beta)
        self.Wh = [rotate_mpo(mpo, b) for b in self.beta]
        self.Wn = [rotate_mpo(identity_mpo(mps.K), b) for b in self.beta]
        K = mps.K
        G = len(self.beta)
        self.Lh = [[None] * (K + 1) for _ in range(G)]
        self.Ln = [[None] * (K + 1) for _ in range(G)]
        self.Rh = [[None] * (K + 1) for _ in range(G)]
        self.Rn = [[None] * (K + 1) for _ in range(G)]
        for g in range(G):
            self.Lh[g][0] = np.ones((1, 1, 1))
            self.Ln[g][0] = np.ones((1, 1, 1))
            self.Rh[g][K] = np.ones((1, 1, 1))
            self.Rn[g][K] = np.ones((1, 1, 1))

    def build_left(self, upto: int):
        for i in range(1, upto + 1):
            self.update_left(i - 1)

    def build_right(self, downto: int):
        for i in range(self.mps.K - 1, downto - 1, -1):
            self.update_right(i)

    def update_left(self, site: int):
        """L at bond site+1 from L at bond site and A[site]."""
        A = self.mps.A[site]
        for g in range(len(self.beta)):
            self.Lh[g][site + 1] = left_env_update(self.Lh[g][site], A, self.Wh[g][site])
            self.Ln[g][site + 1] = left_env_update(self.Ln[g][site], A, self.Wn[g][site])

    def update_right(self, site: int):
        """R at bond site from R at bond site+1 and A[site]."""
        A = self.mps.A[site]
        for g in range(len(self.beta)):
            self.Rh[g][site] = right_env_update(self.Rh[g][site + 1], A, self.Wh[g][site])
            self.Rn[g][site] = right_env_update(self.Rn[g][site + 1], A, self.Wn[g][site])

    # ---- the projected action -------------------------------------------------------------

    def apply(self, x, k, which=("h", "n"), screen=0.0):
        """(y, z) = (H_eff x, N_eff x) at sites (k, k+1); x has shape (Dl, 4, 4, Dr).  With
        screen > 0 the environments are first screened (``screen_environment``): the M-sector
        screening of Sec. 2.3.1's closing paragraph, an approximation."""
        ql, qr = self.mps.labels[k], self.mps.labels[k + 2]
        mask = two_site_mask(ql, qr)
        out = []
        for kind in which:
            acc = np.zeros_like(x)
            for g, cg in enumerate(self.c):
                if kind == "h":
                    L, R = self.Lh[g][k], self.Rh[g][k + 2]
                    W1, W2 = self.Wh[g][k], self.Wh[g][k + 1]
                else:
                    L, R = self.Ln[g][k], self.Rn[g][k + 2]
                    W1, W2 = self.Wn[g][k], self.Wn[g][k + 1]
                if screen > 0.0:
                    L = screen_environment(L, ql, ql, screen)
                    R = screen_environment(R, qr, qr, screen)
                T = np.einsum("awc,ctid->awtid", L, x)
                T = np.einsum("awtid,wvst->avsid", T, W1)
                T = np.einsum("avsid,vuji->asjud", T, W2)
                acc += cg * np.einsum("asjud,bud->asjb", T, R)
            out.append(np.where(mask, acc, 0.0))
        return tuple(out)

    def apply_rows(self, x, k, rows, which=("h", "n")):
        """The same projected action restricted to the bra rows ``rows`` of the left bond
        (a subset of output entries, for checks at sizes where the full output is too slow)."""
        ql, qr = self.mps.labels[k], self.mps.labels[k + 2]
        mask = two_site_mask(ql, qr)[rows]
        out = []
        for kind in which:
            acc = np.zeros((len(rows),) + x.shape[1:])
            for g, cg in enumerate(self.c):
                if kind == "h":
                    L, R = self.Lh[g][k][rows], self.Rh[g][k + 2]
                    W1, W2 = self.Wh[g][k], self.Wh[g][k + 1]
                else:
                    L, R = self.Ln[g][k][rows], self.Rn[g][k + 2]
                    W1, W2 = self.Wn[g][k], self.Wn[g][k + 1]
                T = np.einsum("awc,ctid->awtid", L, x)
                T = np.einsum("awtid,wvst->avsid", T, W1)
                T = np.einsum("avsid,vuji->asjud", T, W2)
                acc += cg * np.einsum("asjud,bud->asjb", T, R)
            out.append(np.where(mask, acc, 0.0))
        return tuple(out)

    def diagonal(self, k):
        """Diagonals of H_eff and N_eff at sites (k, k+1) (preconditioner input)."""
        ql, qr = self.mps.labels[k], self.mps.labels[k + 2]
        mask = two_site_mask(ql, qr)
        out = []
        for kind in ("h", "n"):
            acc = 0.0
            for g, cg in enumerate(self.c):
                if kind == "h":
                    L, R = self.Lh[g][k], self.Rh[g][k + 2]
                    W1, W2 = self.Wh[g][k], self.Wh[g][k + 1]
                else:
                    L, R = self.Ln[g][k], self.Rn[g][k + 2]
                    W1, W2 = self.Wn[g][k], self.Wn[g][k + 1]
                Ld = np.einsum("awa->aw", L)
                Rd = np.einsum("bub->bu", R)
                W1d = np.einsum("wvss->wvs", W1)
                W2d = np.einsum("vujj->vuj", W2)
                acc = acc + cg * np.einsum("aw,wvs,vuj,bu->asjb", Ld, W1d, W2d, Rd)
            out.append(np.where(mask, acc, 0.0))
        return tuple(out)

    def metric_blocks(self, k, max_dim=None):
        """The diagonal blocks of N_eff at sites (k, k+1) in the (N, M)-allowed entries of the
        two-site tensor, one block per (n of the left bond index, n(s1), n(s2)): a list of
        (positions in the flattened masked vector, dense block).  Block entries are
        sum_g c_g LN_g[a, a'] rN_g[s1, s1'] rN_g[s2, s2'] RN_g[b, b'] (the identity MPO rotated
        by beta_g has bond dimension 1)."""
        ql, qr = self.mps.labels[k], self.mps.labels[k + 2]
        mask = two_site_mask(ql, qr)
        ia, i1, i2, ib = np.nonzero(mask)
        nloc = LOCAL_Q[:, 0]
        key = np.stack([ql[ia, 0], nloc[i1], nloc[i2]], axis=1)
        out = []
        for kk in sorted(set(map(tuple, key))):
            pos = np.nonzero(np.all(key == kk, axis=1))[0]
            if max_dim is not None and len(pos) > max_dim:
                continue
            a, s1, s2, b = ia[pos], i1[pos], i2[pos], ib[pos]
            blk = np.zeros((len(pos), len(pos)))
            for g, cg in enumerate(self.c):
                L = self.Ln[g][k][:, 0, :]
                R = self.Rn[g][k + 2][:, 0, :]
                r1 = self.Wn[g][k][0, 0]
                r2 = self.Wn[g][k + 1][0, 0]
                blk += cg * L[np.ix_(a, a)] * r1[np.ix_(s1, s1)] * r2[np.ix_(s2, s2)] * R[np.ix_(b, b)]
            out.append((pos, blk))
        return out

    def two_site(self, k):
        return np.einsum("asc,cjb->asjb", self.mps.A[k], self.mps.A[k + 1])

    def energy(self, k):
        """E and <P> at the orthogonality centre (sites k, k+1): Eq. efunctional."""
        x = self.two_site(k)
        y, z = self.apply(x, k)
        return float(np.vdot(x, y) / np.vdot(x, z)), float(np.vdot(x, z) / np.vdot(x, x))


# ---- generalised Davidson -------------------------------------------------------------------

@dataclass
class DavidsonResult:
    theta: float
    x: np.ndarray
    iterations: int
    converged: bool
    residual: float


def davidson(apply_hn, x0, diag_h, diag_n, mask, tol_r=1e-6, tol_theta=1e-10,
             max_sub=20, max_iter=200, eps_metric=1e-12, clamp=1e-4,
             precond="diag", apply_n=None, cg_steps=5, metric_blocks=None,
             metric_shift=METRIC_SHIFT, constraints=None) -> DavidsonResult:
    """Lowest eigenpair of H x = theta N x with N positive semi-definite.

    Basis V Euclidean-orthonormal (classical Gram-Schmidt applied twice); Ritz problem
    h c = theta n c solved by canonical orthogonalisation of n (eigenvalues below
    eps_metric * max dropped); x = V c with x^T N x = 1; residual r = H x - theta N x;
    correction t = -r / (diag H - theta diag N), the denominator clamped to |.| >= clamp
    (precond="diag"), or t = cg_steps conjugate-gradient steps on N t = r from t = 0
    (precond="metric", an approximate N^+ r; needs ``apply_n``), or
    t = (N_b + metric_shift I)^-1 r on every diagonal block N_b of N given in ``metric_blocks``
    (precond="metric_block"; from Projected.metric_blocks: N is block-diagonal, so this is the
    inverse of N shifted by metric_shift, which keeps directions of N-norm down to ~metric_shift;
    entries of blocks left out keep the diagonal correction);
    restart from [x, previous x] when the basis reaches max_sub; converged when
    ||r|| < tol_r and |theta - theta_prev| < tol_theta.  ``constraints`` (orthonormal columns V over
    the masked entries, or None): the start vector and every correction are projected with
    Q = 1 - V V^T, so the solve stays in the range of Q (excited states, Eq. orthoB)."""
    shape = x0.shape
    sel = mask.reshape(-1)
    v = x0.reshape(-1)[sel]
    dh, dn = diag_h.reshape(-1)[sel], diag_n.reshape(-1)[sel]

    def op(u):
        full = np.zeros(sel.shape[0])
        full[sel] = u
        y, z = apply_hn(full.reshape(shape))
        return y.reshape(-1)[sel], z.reshape(-1)[sel]

    def op_n(u):
        full = np.zeros(sel.shape[0])
        full[sel] = u
        return apply_n(full.reshape(shape)).reshape(-1)[sel]

    Qc = (lambda u: u - constraints @ (constraints.T @ u)) if constraints is not None else (lambda u: u)
    v = Qc(Qc(v))
    V = (v / np.linalg.norm(v))[:, None]
    y, z = op(V[:, 0])
    HV, NV = y[:, None], z[:, None]
    theta_prev = np.inf
    x_prev = None
    theta, x, rn = np.inf, V[:, 0], np.inf
    for it in range(1, max_iter + 1):
        h = V.T @ HV
        n = V.T @ NV
        h = 0.5 * (h + h.T)
        n = 0.5 * (n + n.T)
        mu, Q = np.linalg.eigh(n)
        # unit basis vectors and |N| <= 1: an n-eigenvalue below METRIC_FLOOR is numerically zero
        keep = (mu > eps_metric * mu.max()) & (mu > METRIC_FLOOR)
        if mu.max() <= 0 or not keep.any():
            raise FloatingPointError("singular metric")
        X = Q[:, keep] / np.sqrt(mu[keep])
        hp = X.T @ h @ X
        th, C = np.linalg.eigh(0.5 * (hp + hp.T))
        theta = th[0]
        c = X @ C[:, 0]
        x = V @ c
        hx, nx = HV @ c, NV @ c
        r = Qc(hx - theta * nx)  # with constraints: the residual within the range of Q
        rn = np.linalg.norm(r)
        if rn < tol_r and abs(theta - theta_prev) < tol_theta:
            full = np.zeros(sel.shape[0])
            full[sel] = x
            return DavidsonResult(theta, full.reshape(shape), it, True, rn)
        theta_prev = theta
        if precond == "metric":
            t = _cg_metric(lambda u: op_n(u), r, cg_steps)
        elif precond == "metric_block":
            den = dh - theta * dn
            den = np.where(np.abs(den) < clamp, np.where(den < 0, -clamp, clamp), den)
            t = -r / den
            for pos, blk in metric_blocks:
                t[pos] = np.linalg.solve(blk + metric_shift * np.eye(len(pos)), r[pos])
        else:
            den = dh - theta * dn
            den = np.where(np.abs(den) < clamp, np.where(den < 0, -clamp, clamp), den)
            t = -r / den
        if V.shape[1] >= max_sub:
            basis = [x] if x_prev is None else [x, x_prev]
            B = np.stack(basis, axis=1)
            # coefficients of the restart vectors in the old basis
            Cb = V.T @ B
            Qb, _ = np.linalg.qr(Cb)
            V, HV, NV = V @ Qb, HV @ Qb, NV @ Qb
        t = Qc(t)
        for _ in range(2):
            t = t - V @ (V.T @ t)
        t = Qc(t)
        tn = np.linalg.norm(t)
        if tn < 1e-14:
            t = Qc(r.copy())
            for _ in range(2):
                t = t - V @ (V.T @ t)
            tn = np.linalg.norm(t)
            if tn < 1e-14:
                break
        t = t / tn
        y, z = op(t)
        V = np.concatenate([V, t[:, None]], axis=1)
        HV = np.concatenate([HV, y[:, None]], axis=1)
        NV = np.concatenate([NV, z[:, None]], axis=1)
        x_prev = x
    full = np.zeros(sel.shape[0])
    full[sel] = x
    return DavidsonResult(theta, full.reshape(shape), max_iter, False, rn)


def min_norm_representative(x, nx, metric_blocks, shift=METRIC_SHIFT):
    """The two-site vector is defined only modulo ker N_eff (several results are correct); before
    decimation the metric_block form takes the representative x' = (N + shift I)^-1 N x, built
    from N x (masked, flattened) block by block: x' keeps every component of x along directions
    of N-norm well above ``shift`` and drops the (near-)null ones, which P V x does not see but
    which would otherwise dominate the singular values of x.  Entries of blocks left out of
    ``metric_blocks`` keep x."""
    out = np.array(x, dtype=float, copy=True)
    for pos, blk in metric_blocks:
        out[pos] = np.linalg.solve(blk + shift * np.eye(len(pos)), nx[pos])
    return out


def _cg_metric(apply_n, r, steps):
    """Plain conjugate gradients on N t = r, started from t = 0."""
    t = np.zeros_like(r)
    res = r.copy()
    p = res.copy()
    rr = res @ res
    for _ in range(steps):
        ap = apply_n(p)
        pap = p @ ap
        if pap <= 0.0 or rr == 0.0:
            break
        a = rr / pap
        t += a * p
        res -= a * ap
        rr_new = res @ res
        p = res + (rr_new / rr) * p
        rr = rr_new
    return t


# ---- decimation ---------------------------------------------------------------------------

TIE_RTOL = 1e-10
DROP_ABS = 1e-7  # dropped weight per singular value < 1e-14 (|x| = 1)


def ordered_truncation(values, labels, D):
    """Keep the D largest of ``values`` (singular values).  Sorted descending; values
    within TIE_RTOL * max of their sorted predecessor form a tie cluster, ordered inside by
    (n, 2m, index-in-block) ascending; values below DROP_ABS are dropped.
    ``labels`` holds (n, 2m, index) per value.  Returns the kept positions."""
    values = np.asarray(values)
    if len(values) == 0:
        return []
    order = sorted(range(len(values)), key=lambda j: -values[j])
    vmax = values[order[0]]
    clusters, cur = [], [order[0]]
    for j in order[1:]:
        if values[cur[-1]] - values[j] <= TIE_RTOL * vmax:
            cur.append(j)
        else:
            clusters.append(cur)
            cur = [j]
    clusters.append(cur)
    ranked = []
    for cl in clusters:
        ranked.extend(sorted(cl, key=lambda j: tuple(labels[j])))
    ranked = [j for j in ranked if values[j] >= DROP_ABS]
    return ranked[:D]


def decimate(x, ql, qr, D, move_right: bool):
    """Split x[a, s1, s2, b] by SVD per middle label q(a)+q(s1) and truncate.
    Returns (A_left, A_right, labels_mid, discarded_weight)."""
    Dl, Dr = ql.shape[0], qr.shape[0]
    x = x / np.linalg.norm(x)
    X = x.reshape(Dl * 4, 4 * Dr)
    qrow = (ql[:, None, :] + LOCAL_Q[None, :, :]).reshape(-1, 2)
    qcol = (qr[None, :, :] - LOCAL_Q[:, None, :]).reshape(-1, 2)
    mids = sorted(set(map(tuple, qrow)) & set(map(tuple, qcol)))
    svals, tags, parts = [], [], []
    for q in mids:
        rows = np.nonzero(np.all(qrow == q, axis=1))[0]
        cols = np.nonzero(np.all(qcol == q, axis=1))[0]
        U, S, Vt = np.linalg.svd(X[np.ix_(rows, cols)], full_matrices=False)
        parts.append((q, rows, cols, U, S, Vt))
        for j, s in enumerate(S):
            svals.append(s)
            tags.append((q[0], q[1], j))
    keep = ordered_truncation(svals, tags, D)
    kept = {}
    for j in keep:
        n, m, idx = tags[j]
        kept.setdefault((n, m), []).append(idx)
    keepset = set(keep)
    disc = float(sum(s * s for j, s in enumerate(svals) if j not in keepset))
    newl, blocksL, blocksR = [], [], []
    for (q, rows, cols, U, S, Vt) in parts:
        if q not in kept:
            continue
        idx = sorted(kept[q])
        bl = np.zeros((Dl * 4, len(idx)))
        br = np.zeros((len(idx), 4 * Dr))
        if move_right:
            bl[rows] = U[:, idx]
            br[:, cols] = S[idx, None] * Vt[idx]
        else:
            bl[rows] = U[:, idx] * S[None, idx]
            br[:, cols] = Vt[idx]
        blocksL.append(bl)
        blocksR.append(br)
        newl.extend([q] * len(idx))
    Al = np.concatenate(blocksL, axis=1)
    Ar = np.concatenate(blocksR, axis=0)
    labels_mid = np.array(newl, dtype=np.int64).reshape(-1, 2)
    return Al.reshape(Dl, 4, -1), Ar.reshape(-1, 4, Dr), labels_mid, disc


# ---- sweeps -----------------------------------------------------------------------------

@dataclass
class SweepLog:
    theta: list = field(default_factory=list)
    iterations: list = field(default_factory=list)
    discarded: list = field(default_factory=list)
    sweep_energy: list = field(default_factory=list)


def sweep_schedule(K):
    """One sweep: left-to-right steps k = 0..K-3 (centre moves right), then right-to-left
    steps k = K-2..0 (centre moves left); 2K-3 two-site steps, centre back on site 0."""
    return [(k, True) for k in range(K - 2)] + [(k, False) for k in range(K - 2, -1, -1)]


def two_site_step(P: Projected, k: int, move_right: bool, D: int, log: SweepLog, **dav):
    mps = P.mps
    x0 = P.two_site(k)
    ql, qr = mps.labels[k], mps.labels[k + 2]
    mask = two_site_mask(ql, qr)
    dh, dn = P.diagonal(k)
    blocks = None
    if dav.get("precond") == "metric_block":
        blocks = P.metric_blocks(k, dav.pop("metric_max_dim", None))
        dav = dict(dav, metric_blocks=blocks)
    res = davidson(lambda v: P.apply(v, k), x0, dh, dn, mask,
                   apply_n=lambda v: P.apply(v, k, which=("n",))[0], **dav)
    x = res.x
    if blocks is not None:
        sel = mask.reshape(-1)
        nx = P.apply(x, k, which=("n",))[0].reshape(-1)[sel]
        full = np.zeros(mask.size)
        full[sel] = min_norm_representative(x.reshape(-1)[sel], nx, blocks, dav.get("metric_shift", METRIC_SHIFT))
        x = full.reshape(mask.shape)
    Al, Ar, lm, disc = decimate(x, ql, qr, D, move_right)
    mps.A[k], mps.A[k + 1] = Al, Ar
    mps.labels[k + 1] = lm
    if move_right:
        P.update_left(k)
        mps.center = k + 1
    else:
        P.update_right(k + 1)
        mps.center = k
    log.theta.append(res.theta)
    log.iterations.append(res.iterations)
    log.discarded.append(disc)
    return res


def run_sweeps(P: Projected, D: int, n_sweeps: int, log: SweepLog | None = None, **dav) -> SweepLog:
    """Two-site sweeps from an MPS with its centre on site 0 and right environments built."""
    log = log or SweepLog()
    K = P.mps.K
    for _ in range(n_sweeps):
        for k, mr in sweep_schedule(K):
            two_site_step(P, k, mr, D, log, **dav)
        log.sweep_energy.append(log.theta[-1])
    return log


def prepare(labels, tensors, mpo, twoS, twoM, n_beta) -> Projected:
    """Right-canonicalise a raw MPS and build all right environments (centre on site 0)."""
    mps = right_canonicalize(labels, tensors)
    P = Projected(mps, mpo, twoS, twoM, n_beta)
    P.build_right(2)
    return P


def to_full_vector(mps: MPS) -> np.ndarray:
    """Contract the MPS to the 4^K Fock tensor (site 0 most significant)."""
    cur = mps.A[0][0]  # (4, D1)
    for A in mps.A[1:]:
        cur = np.einsum("Sa,atb->Stb", cur, A).reshape(-1, A.shape[2])
    return cur[:, 0]
