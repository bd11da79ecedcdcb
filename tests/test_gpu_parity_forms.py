"""Parity with the oracle of the parts of the path the benchmark times beyond the FP64 action:
the reduced-precision (TF32 / 3xTF32 tensor-core) action at full size, and the truncating
decimation (Sec. 2.3.1: SVD of the two-site tensor per middle label, keep the D largest).

Reduced-precision bound, element by element (derived from the split, not fitted):
  |y_gpu - y| <= (g_A + g_C + g_A g_C) * y_abs,
  y_abs = sum_g |c_g| |L_g| |x| |W_k| |W_k+1| |R_g| (the same network on absolute values),
  g_X = u + K_X 2^-24 for the GEMM phases A (L x, reduction length K_A = largest label of bond k)
  and C (T3 R^T, K_C = channels x largest N-group of bond k+2), FP32 accumulation;
  u = 2 * 2^-11 + 2^-21 per product for TF32 (both operands rounded to 10 mantissa bits),
  u = 4 * 2^-22 for 3xTF32 (the dropped lo*lo term and the rounding of lo).
Phase B (the MPO legs) is FP64.  z = N_eff x is always FP64 and is compared at 1e-10.
"""
import numpy as np
import pytest

from oracle import mpo as M, mps as S
from paper_1703_04789_gb300 import inputs
from tests.gpu_util import masked_random_two_site, require_gpu


def _abs_rows(P, x, k, rows):
    """sum_g |c_g| |L_g| |x| |W_k| |W_k+1| |R_g| on the bra rows `rows` (H network)."""
    acc = 0.0
    xa = np.abs(x)
    for g, cg in enumerate(P.c):
        L = np.abs(P.Lh[g][k][rows])
        R = np.abs(P.Rh[g][k + 2])
        W1, W2 = np.abs(P.Wh[g][k]), np.abs(P.Wh[g][k + 1])
        T = np.einsum("awc,ctid->awtid", L, xa)
        T = np.einsum("awtid,wvst->avsid", T, W1)
        T = np.einsum("avsid,vuji->asjud", T, W2)
        acc = acc + abs(cg) * np.einsum("asjud,bud->asjb", T, R)
    return acc


def _max_group(q):
    ns, counts = np.unique(q[:, 0], return_counts=True)
    return int(counts.max())


def _max_label(q):
    _, counts = np.unique(q, axis=0, return_counts=True)
    return int(counts.max())


@pytest.mark.gpu
@pytest.mark.parametrize("twoM,twoS", [(0, 0), (2, 2)])
def test_reduced_precision_action_matches_oracle_full_size(twoM, twoS):
    """Hubbard L=24, half filling, D=256, n_beta=8, middle site, with the fast form's settings
    (autotuned tiles, pre-split tensor-core operands): sampled bra rows of y against the oracle
    within the split bound, z at FP64 accuracy, for TF32 and 3xTF32 on the stacked tcgen05 GEMM and
    for 3xTF32 on the warp-level mma.sync kernel."""
    require_gpu()
    from paper_1703_04789_gb300 import Spmps
    L, N, D, G, U = 24, 24, 256, 8, 4.0
    labels, tens = inputs.random_mps(L, N, twoM, D, 2)
    P = S.prepare(labels, tens, M.hubbard_mpo(L, 1.0, U), twoS, twoM, G)
    k = L // 2 - 1
    P.build_left(k)
    ql, qr = P.mps.labels[k], P.mps.labels[k + 2]
    rng = np.random.default_rng(17)
    x = masked_random_two_site(ql, qr, rng)
    rows = sorted(set(rng.choice(ql.shape[0], size=10, replace=False).tolist() + [0, ql.shape[0] - 1]))
    y_ref, z_ref = P.apply_rows(x, k, rows)
    y_abs = _abs_rows(P, x, k, rows)
    mask = S.two_site_mask(ql, qr)[rows]
    K_A = _max_label(ql)
    K_C = 6 * _max_group(qr)
    cases = [("3xtf32", 4 * 2.0 ** -22, "tcgen05"), ("tf32", 2 * 2.0 ** -11 + 2.0 ** -21, "tcgen05"),
             ("3xtf32", 4 * 2.0 ** -22, "mma_sync")]
    for prec, u, kern in cases:
        dev = Spmps(L, N, twoM, twoS, G, D, precision=prec, autotune=True, tensor_core_kernel=kern)
        dev.set_hubbard(1.0, U)
        dev.set_mps(P.mps.labels, P.mps.A, center=0)
        lay = dev.x_layout(k)
        yv, zv = dev.apply_heff_host(k, dev.pack(x, lay, ql, qr))
        y = dev.unpack(yv, lay, ql, qr)[rows]
        z = dev.unpack(zv, lay, ql, qr)[rows]
        dev.close()
        gA, gC = u + K_A * 2.0 ** -24, u + K_C * 2.0 ** -24
        bound = (gA + gC + gA * gC) * y_abs
        err = np.abs(y - y_ref)
        assert np.all(err[mask] <= bound[mask] + 1e-300), (prec, kern, float((err / np.maximum(bound, 1e-300))[mask].max()))
        assert err[mask].max() > 0.0  # the tensor-core path ran
        assert np.abs(z - z_ref).max() <= 1e-10 * max(1.0, np.abs(z_ref).max())


def _decimation_case(L, N, Dm, Dh, G, k, move_right, seed):
    from paper_1703_04789_gb300 import Spmps
    labels, tens = inputs.random_mps(L, N, 0, Dm, seed)
    x0 = np.einsum("asc,cjb->asjb", tens[k], tens[k + 1])
    x0 = np.where(S.two_site_mask(labels[k], labels[k + 2]), x0, 0.0)
    Al, Ar, lm, disc = S.decimate(x0, labels[k], labels[k + 2], Dh, move_right)
    # one Davidson iteration returns x proportional to the current two-site tensor, so the step
    # decimates exactly A[k] A[k+1] of the loaded (non-canonical) MPS to Dh states
    dev = Spmps(L, N, 0, 0, G, Dh, dav_max_iter=1)
    dev.set_hubbard(1.0, 4.0)
    dev.set_mps(labels, tens, center=k if move_right else k + 1)
    dev.optimize_step(k, move_right, allow_not_converged=True)
    disc_gpu = dev.stats()["discarded_weight"]
    lab2, ts2, _ = dev.get_mps()
    dev.close()
    return (Al, Ar, lm, disc), (ts2[k], ts2[k + 1], lab2[k + 1], disc_gpu)


@pytest.mark.gpu
@pytest.mark.parametrize("L,N,Dm,Dh,G,k,move_right,seed", [
    (8, 8, 32, 12, 5, 3, True, 1),     # the L=8, D=32 workload's middle bond, truncated to 12
    (8, 8, 32, 20, 5, 2, False, 3),
    (24, 24, 256, 128, 8, 11, True, 2),  # an L=24, D=256 middle bond, truncated to 128
])
def test_truncating_decimation_matches_oracle(L, N, Dm, Dh, G, k, move_right, seed):
    """The kept (n, 2m) multiset, the kept singular values (1e-10), the discarded weight (1e-10)
    and the truncated two-site tensor (1e-9) equal the oracle's SVD truncation of the same x."""
    require_gpu()
    (Al, Ar, lm, disc), (Ag, Bg, lg, disc_g) = _decimation_case(L, N, Dm, Dh, G, k, move_right, seed)
    assert sorted(map(tuple, lg.tolist())) == sorted(map(tuple, lm.tolist()))
    assert lg.shape[0] == lm.shape[0] <= Dh
    if move_right:
        s_ref = np.linalg.norm(Ar.reshape(Ar.shape[0], -1), axis=1)
        s_gpu = np.linalg.norm(Bg.reshape(Bg.shape[0], -1), axis=1)
    else:
        s_ref = np.linalg.norm(Al.reshape(-1, Al.shape[2]), axis=0)
        s_gpu = np.linalg.norm(Ag.reshape(-1, Ag.shape[2]), axis=0)
    assert np.abs(np.sort(s_gpu) - np.sort(s_ref)).max() < 1e-10
    assert abs(disc_g - disc) < 1e-10
    x_ref = np.einsum("asc,cjb->asjb", Al, Ar)
    x_gpu = np.einsum("asc,cjb->asjb", Ag, Bg)
    assert np.abs(x_gpu - x_ref).max() < 1e-9
