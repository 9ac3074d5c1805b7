"""CPU oracle of the Taylor shift by one -- TEST INFRASTRUCTURE ONLY.

Only tests/ and the oracle leg of bench.py may import this module.  The CUDA
library never imports it; the two share no code.

The paper's application (§1, real root isolation) shifts polynomials by one.
g(x) = f(x + 1) has, by the binomial theorem applied to each f_i (x + 1)^i,
the coefficients

    g_k = sum_{i=k}^{n-1} C(i, k) f_i,

which is what this module computes, with Python's own integers.  The
binomials C(i, k) for fixed k and growing i follow
C(i + 1, k) = C(i, k) (i + 1) / (i + 1 - k), an exact division.
"""
from __future__ import annotations


def taylor_coeff(f: list[int], k: int) -> int:
    """g_k = sum_{i >= k} C(i, k) f_i for g(x) = f(x + 1)."""
    n = len(f)
    total = 0
    c = 1  # C(k, k)
    for i in range(k, n):
        total += c * f[i]
        c = c * (i + 1) // (i + 1 - k)
    return total


def taylor_shift1(f: list[int]) -> list[int]:
    """All coefficients of f(x + 1) (O(n^2) big-integer products: small n)."""
    return [taylor_coeff(f, k) for k in range(len(f))]


def taylor_coeffs(f: list[int], ks) -> list[int]:
    """Coefficients g_k, k in ks, each computed on its own."""
    return [taylor_coeff(f, int(k)) for k in ks]
