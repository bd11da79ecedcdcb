"""Quadrature for the spin projector (oracle; test infrastructure only).

Sec. 2.2, Eq. PSMM: P^S_MM = (2S+1)/2 * int_0^pi sin(b) d^S_MM(b) exp(-i b S_y) db.
Eq. pmpo: with x = cos(b) this becomes a Gauss-Legendre sum over g of
w_g d^S_MM(b_g) exp(-i b_g S_y).  Reading of the paper: the prefactor (2S+1)/2 of Eq. PSMM
is folded into the weights, so that sum_g c_g = <P> of a pure spin-S state equals 1.
Eq. exactQuadrature: the rule is exact when N_g >= ceil((Omega_max/2 + S + 1) / 2).
"""
from __future__ import annotations

from math import factorial, ceil

import numpy as np


def gauss_legendre(n: int) -> tuple[np.ndarray, np.ndarray]:
    """Nodes and weights of the n-point Gauss-Legendre rule on [-1, 1] (library routine)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


def wigner_small_d(two_j: int, two_mp: int, two_m: int, beta: float) -> float:
    """Wigner's small-d element d^j_{m'm}(beta) from Wigner's explicit sum
    (j, m', m given doubled, so half-integers are exact)."""
    if (two_j + two_mp) % 2 or (two_j + two_m) % 2 or abs(two_mp) > two_j or abs(two_m) > two_j:
        raise ValueError("bad angular momentum labels")
    jpmp = (two_j + two_mp) // 2
    jmmp = (two_j - two_mp) // 2
    jpm = (two_j + two_m) // 2
    jmm = (two_j - two_m) // 2
    mpmm = (two_mp - two_m) // 2  # m' - m
    c = np.cos(beta / 2.0)
    s = np.sin(beta / 2.0)
    pref = np.sqrt(float(factorial(jpmp) * factorial(jmmp) * factorial(jpm) * factorial(jmm)))
    total = 0.0
    for k in range(0, two_j + 1):
        a1 = jpm - k
        a2 = mpmm + k
        a3 = jmmp - k
        if a1 < 0 or a2 < 0 or a3 < 0:
            continue
        den = factorial(a1) * factorial(k) * factorial(a2) * factorial(a3)
        sign = -1.0 if (mpmm + k) % 2 else 1.0
        total += sign / den * c ** (a1 + a3) * s ** (a2 + k)
    return pref * total


def omega_max(K: int, N: int, twoM: int) -> int:
    """Maximal seniority of Eq. exactQuadrature."""
    na, nb = (N + twoM) // 2, (N - twoM) // 2
    return min(na, K - nb) + min(nb, K - na)


def n_exact(K: int, N: int, twoM: int, twoS: int) -> int:
    """Smallest number of Gauss-Legendre points for which Eq. pmpo is exact
    (Eq. exactQuadrature); with doubled S the degree bound is (Omega_max + 2S)/2."""
    deg2 = omega_max(K, N, twoM) + twoS  # twice the polynomial degree in x
    return int(ceil((deg2 / 2.0 + 1.0) / 2.0))


def projector_quadrature(twoS: int, twoM: int, n_beta: int):
    """Angles beta_g, coefficients c_g = (2S+1)/2 * w_g * d^S_MM(beta_g), and the
    cos/sin of beta_g/2 that enter the site rotation of Eq. expSy."""
    x, w = gauss_legendre(n_beta)
    beta = np.arccos(x)
    d = np.array([wigner_small_d(twoS, twoM, twoM, b) for b in beta])
    c = 0.5 * (twoS + 1) * w * d
    return beta, c


def site_rotation(beta: float) -> np.ndarray:
    """Eq. expSy: the 4x4 matrix of exp(-i beta S_y,k) in the basis {0, b, a, ab}."""
    c, s = np.cos(beta / 2.0), np.sin(beta / 2.0)
    r = np.eye(4)
    r[1, 1] = c
    r[1, 2] = s
    r[2, 1] = -s
    r[2, 2] = c
    return r
