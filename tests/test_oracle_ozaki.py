"""Pins of the oracle's split-product GEMM (oracle/ozaki.py) against exact arithmetic.

The scheme (error-free splitting into exact small-integer products, Ozaki et al. 2012) must give
the exact product whenever every partial product is representable, and otherwise stay within its
a-priori bound of the exact rational product.  A dropped level, a wrong digit shift or a wrong
scale exponent breaks the exact cases below.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import ozaki as Z


def _exact(A, B):
    M, K = A.shape
    N = B.shape[1]
    out = np.empty((M, N), dtype=object)
    Af = [[Fraction(float(A[i, k])) for k in range(K)] for i in range(M)]
    Bf = [[Fraction(float(B[k, j])) for j in range(N)] for k in range(K)]
    for i in range(M):
        for j in range(N):
            out[i, j] = sum((Af[i][k] * Bf[k][j] for k in range(K)), Fraction(0))
    return out


def test_digits_reconstruct_entries_near_the_line_maximum():
    rng = np.random.default_rng(1)
    X = rng.uniform(0.5, 1.0, size=(6, 32)) * np.where(rng.random((6, 32)) < 0.5, -1.0, 1.0)
    X *= 2.0 ** rng.integers(-3, 1, size=(6, 32))  # within 2^3 of the row maximum: 56 bits hold them
    e = Z.chunk_exponents(X, axis=1)
    D = Z.digits(X, e[:, None])
    assert np.abs(D).max() <= 255
    rec = sum(np.ldexp(D[p].astype(np.float64), (e[:, None] - 8 * (p + 1)).astype(np.int32)) for p in range(7))
    assert np.array_equal(rec, X)


@pytest.mark.parametrize("K", [1, 31, 32, 33, 100])
def test_integer_matrices_are_exact(K):
    """Integer entries below 2^20: every digit product and every sum is exact, so the result is
    the integer product (bit-exact), whatever the chunking."""
    rng = np.random.default_rng(K)
    A = rng.integers(-2 ** 20, 2 ** 20, size=(9, K)).astype(np.float64)
    B = rng.integers(-2 ** 20, 2 ** 20, size=(K, 7)).astype(np.float64)
    ref = A.astype(np.int64) @ B.astype(np.int64)
    assert np.array_equal(Z.matmul(A, B), ref.astype(np.float64))


def test_identity_and_zero():
    rng = np.random.default_rng(3)
    B = rng.uniform(1.0, 2.0, size=(40, 5))  # one binade per column: exact digits
    assert np.array_equal(Z.matmul(np.eye(40), B), B)
    assert np.array_equal(Z.matmul(np.zeros((3, 40)), B), np.zeros((3, 5)))
    assert np.array_equal(Z.matmul(np.eye(40)[:4], np.zeros((40, 2))), np.zeros((4, 2)))


def test_worst_case_digits_keep_level_sums_exact_in_fp32():
    """All digits 255 (entries just below the line's power of two): the level sums reach their
    largest size and must stay below 2^24 (asserted inside), the result within the bound."""
    x = 1.0 - 2.0 ** -53
    A = np.full((4, 32), x)
    B = np.full((32, 3), -x)
    C = Z.matmul(A, B)
    ex = _exact(A, B)
    err = np.array([[abs(Fraction(float(C[i, j])) - ex[i, j]) for j in range(3)] for i in range(4)], dtype=float)
    assert np.all(err <= Z.error_bound(A, B))


@pytest.mark.parametrize("seed,spread", [(4, 0), (5, 6), (6, 30)])
def test_random_products_within_the_bound_of_the_exact_product(seed, spread):
    """Random FP64 entries over 2^spread binades, K spanning three chunks and a ragged tail: the
    error against the exact rational product stays within the a-priori bound; with entries of
    one size the bound is within a few times the FP64 bound K u |A| |B|."""
    rng = np.random.default_rng(seed)
    M, K, N = 5, 75, 4
    A = rng.standard_normal((M, K)) * 2.0 ** rng.integers(-spread, 1, size=(M, K))
    B = rng.standard_normal((K, N)) * 2.0 ** rng.integers(-spread, 1, size=(K, N))
    C = Z.matmul(A, B)
    ex = _exact(A, B)
    err = np.array([[abs(Fraction(float(C[i, j])) - ex[i, j]) for j in range(N)] for i in range(M)], dtype=float)
    bnd = Z.error_bound(A, B)
    assert np.all(err <= bnd)
    if spread == 0:
        assert np.all(bnd <= 4 * K * 2.0 ** -53 * (np.abs(A) @ np.abs(B)))


def test_scheme_on_the_action_operands_stays_at_fp64_level():
    """The two GEMM phases of the projected action (Fig. spmpsOpt) on real operands of the path --
    rotated environments and a masked two-site vector of an L=6 Hubbard MPS at the middle site --
    computed by the splitting scheme stay within its bound and within 1e-14 (relative to the
    largest |A| |B| entry) of the FP64 products."""
    from oracle import mpo as M, mps as S
    from paper_1703_04789_gb300 import inputs
    L, N, D, G = 6, 6, 16, 4
    labels, tens = inputs.random_mps(L, N, 0, D, 2)
    P = S.prepare(labels, tens, M.hubbard_mpo(L, 1.0, 4.0), 0, 0, G)
    k = L // 2 - 1
    P.build_left(k)
    ql, qr = P.mps.labels[k], P.mps.labels[k + 2]
    rng = np.random.default_rng(3)
    x = np.where(S.two_site_mask(ql, qr), rng.standard_normal((ql.shape[0], 4, 4, qr.shape[0])), 0.0)
    for g in range(G):
        Lg, Rg = P.Lh[g][k], P.Rh[g][k + 2]
        a, w, c = Lg.shape
        A = Lg.reshape(a * w, c)                 # phase A: (a w) x c times c x (t i d)
        B = x.reshape(c, -1)
        T1 = Z.matmul(A, B)
        ref = A @ B
        scale = (np.abs(A) @ np.abs(B)).max()
        assert np.abs(T1 - ref).max() <= 1e-14 * scale
        # the scheme's bound plus the FP64 reference's own rounding (K u |A| |B|)
        assert np.all(np.abs(T1 - ref) <= Z.error_bound(A, B) + c * 2.0 ** -53 * (np.abs(A) @ np.abs(B)))
        b, u, d = Rg.shape
        T3 = rng.standard_normal((a * 16, u * d))  # phase C: (a s j) x (u d) times (u d) x b
        Rm = Rg.reshape(b, u * d).T
        C = Z.matmul(T3, Rm)
        refc = T3 @ Rm
        assert np.abs(C - refc).max() <= 1e-14 * (np.abs(T3) @ np.abs(Rm)).max()
