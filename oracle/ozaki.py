"""FP64-accurate matrix product from exact small-integer products (oracle; test infrastructure only).

The plain definition of what the library's split-product GEMM reaches is the FP64 matrix product
itself, and the action parity tests compare with that (``mps.apply``).  This module restates the
splitting scheme the library uses, so that its error bound can be checked on the host against
exact rational arithmetic.  The scheme is the error-free splitting of a product into products of
short slices (Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix multiplication
by using fast routines of matrix multiplication and its applications", Numer. Algorithms 59,
2012), in the form that evaluates the slice products on tensor cores with a floating-point
accumulator that stays exact because every partial sum is an integer below 2^24 (Mukunoki,
Ozaki, Ogita and Imamura, "DGEMM using Tensor Cores, and Its Accurate and Reproducible
Versions", ISC 2020).  Steps, for C = A B with A of M x K and B of K x N:

1. K is cut into chunks of ``kchunk`` (32).  Within a chunk, row i of A gets the exponent e_i with
   max_k |a_ik| < 2^e_i (frexp of the row maximum), column j of B likewise f_j.
2. Each entry becomes the integer F = floor(|a| 2^(56 - e_i)) < 2^56 (subnormal entries are taken
   as zero), cut into s = 7 base-256 digits d_1 .. d_7 (d_1 the most significant), each carrying
   the entry's sign: a ~= sign(a) sum_p d_p 2^(-8p) 2^e_i.
3. For every level l = p + q = 2 .. 9 the integer sum v_l = sum_k sum_{p+q=l} a_(p) b_(q) is formed
   (at most 7 pairs; |v_l| <= 32 * 7 * 255^2 < 2^24, so an FP32 accumulator holds it exactly);
   levels above 9 are dropped (below 5 Kc 2^-64 of the scale 2^(e_i + f_j) together).
4. T = sum_{l<=7} v_l 2^(56 - 8l) + floor(v_8 / 2^8) + floor(v_9 / 2^16), an integer below 2^62
   (|v_2| <= 32 * 255^2 < 2^21), and the chunk contributes the FP64 value of T (rounded to
   nearest) times 2^(e_i + f_j - 56); chunks are added in K order in FP64.
"""
from __future__ import annotations

import numpy as np

RHO = 8          # bits per digit
SLICES = 7       # digits per entry (56 bits)
KCHUNK = 32      # reduction length per exact level sum
LEVELS = range(2, SLICES + 3)  # kept levels p + q = 2 .. 9


def chunk_exponents(X: np.ndarray, axis: int) -> np.ndarray:
    """Step 1: e with max |x| < 2^e along ``axis`` (0 for an all-zero line)."""
    m = np.max(np.abs(X), axis=axis)
    _, e = np.frexp(m)
    return np.where(m > 0.0, e, 0).astype(np.int64)


def digits(X: np.ndarray, e: np.ndarray) -> np.ndarray:
    """Step 2: signed digits D[p] (p = 0 .. 6 for d_1 .. d_7) of every entry of X against the
    exponent array e (broadcast to X's shape)."""
    ax = np.abs(X)
    tiny = ax < np.finfo(np.float64).tiny  # zero or subnormal
    F = np.floor(np.ldexp(np.where(tiny, 0.0, ax), (SLICES * RHO - e).astype(np.int32)))
    F = F.astype(np.int64)  # exact: F < 2^56
    sgn = np.where(X < 0.0, -1, 1).astype(np.int64)
    D = np.empty((SLICES,) + X.shape, dtype=np.int64)
    for p in range(1, SLICES + 1):
        D[p - 1] = sgn * ((F >> (SLICES * RHO - RHO * p)) & ((1 << RHO) - 1))
    return D


def chunk_product(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Steps 1-4 for one chunk (A: M x Kc, B: Kc x N, Kc <= KCHUNK)."""
    e = chunk_exponents(A, axis=1)  # per row of A
    f = chunk_exponents(B, axis=0)  # per column of B
    DA = digits(A, e[:, None])
    DB = digits(B, f[None, :])
    T = np.zeros((A.shape[0], B.shape[1]), dtype=np.int64)
    for l in LEVELS:
        v = np.zeros_like(T)
        for p in range(max(1, l - SLICES), min(SLICES, l - 1) + 1):
            v += DA[p - 1] @ DB[l - p - 1]  # exact integer products
        assert np.abs(v).max(initial=0) < 2 ** 24
        sh = SLICES * RHO - RHO * l
        T += v << sh if sh >= 0 else v >> (-sh)  # >> is a floor on int64
    return np.ldexp(T.astype(np.float64), (e[:, None] + f[None, :] - SLICES * RHO).astype(np.int32))


def matmul(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """C = A B by the splitting scheme, chunks of KCHUNK added in K order in FP64."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    C = np.zeros((A.shape[0], B.shape[1]))
    for k0 in range(0, A.shape[1], KCHUNK):
        C = C + chunk_product(A[:, k0:k0 + KCHUNK], B[k0:k0 + KCHUNK, :])
    return C


def error_bound(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A priori bound on |matmul(A, B) - A B| per entry: per chunk, the digit truncation of A and
    B (each below 2^-56 of the line's scale, times Kc), the dropped levels (below Kc 2^-61), the
    two floors (2^-55), all in units of 2^(e_i + f_j); plus the rounding of T and of the running
    FP64 sum (2^-53 per chunk of the absolute partial sums)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    bound = np.zeros((A.shape[0], B.shape[1]))
    run = np.zeros_like(bound)
    u = 2.0 ** -53
    for k0 in range(0, A.shape[1], KCHUNK):
        a, b = A[:, k0:k0 + KCHUNK], B[k0:k0 + KCHUNK, :]
        kc = a.shape[1]
        scale = np.ldexp(1.0, (chunk_exponents(a, 1)[:, None] + chunk_exponents(b, 0)[None, :]).astype(np.int32))
        part = np.abs(a) @ np.abs(b)
        run = run + part
        bound += scale * (2 * kc * 2.0 ** -56 + kc * 2.0 ** -61 + 2.0 ** -55) + 2 * u * (part + run)
    return bound
