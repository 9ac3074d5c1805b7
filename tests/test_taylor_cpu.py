"""Pins of the Taylor-shift oracle (oracle/taylor.py) to what the
mathematics fixes, independent of its own formula:

* f = x^j gives g = (x + 1)^j, whose coefficients are the binomials
  C(j, k) (math.comb, the binomial theorem);
* g(t) = f(t + 1) at integer points t, by Horner's rule on both sides;
* shifting twice equals shifting by two: f(x + 2) at integer points;
* brute force on tiny inputs: expand sum f_i (x + 1)^i by repeated
  multiplication of coefficient lists.
"""
import math

import numpy as np
import pytest

from oracle.taylor import taylor_coeffs, taylor_shift1


def horner(c, t):
    v = 0
    for x in reversed(c):
        v = v * t + x
    return v


@pytest.mark.parametrize("j,n", [(0, 1), (1, 2), (5, 8), (17, 20), (40, 41)])
def test_monomial_gives_binomials(j, n):
    f = [0] * n
    f[j] = 1
    g = taylor_shift1(f)
    assert g == [math.comb(j, k) for k in range(n)]


@pytest.mark.parametrize("n,bits", [(1, 5), (2, 64), (7, 100), (33, 255), (64, 1000)])
def test_evaluation_identity(n, bits):
    rng = np.random.default_rng(n + bits)
    f = [int.from_bytes(rng.bytes((bits + 7) // 8), "little") % (1 << bits) * (1 if rng.random() < 0.5 else -1)
         for _ in range(n)]
    g = taylor_shift1(f)
    for t in (-3, -1, 0, 1, 2, 12345, -(1 << 70)):
        assert horner(g, t) == horner(f, t + 1)
    gg = taylor_shift1(g)
    for t in (0, 5, -7):
        assert horner(gg, t) == horner(f, t + 2)


def test_brute_force_expansion():
    rng = np.random.default_rng(3)
    f = [int(x) for x in rng.integers(-1000, 1000, 9)]
    want = [0] * len(f)
    power = [1]  # (x + 1)^i
    for fi in f:
        for k, c in enumerate(power):
            want[k] += fi * c
        power = [a + b for a, b in zip(power + [0], [0] + power)]
    assert taylor_shift1(f) == want


def test_sampled_coefficients_match_full():
    rng = np.random.default_rng(4)
    f = [int(x) for x in rng.integers(-(1 << 40), 1 << 40, 50)]
    g = taylor_shift1(f)
    ks = [0, 1, 7, 25, 48, 49]
    assert taylor_coeffs(f, ks) == [g[k] for k in ks]
