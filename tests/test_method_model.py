"""A pure-Python model of the paper's method, step by step, checked against
the plain definition c = a*b and against textbook facts -- so every reading
the CUDA path relies on is pinned on the CPU, with no GPU and no library
code:

* split (§2, BivariateRepresentation; reading R1): balanced base-2^M digits
  of the N-bit two's complement, carry rule for j < K-1, top digit absorbing
  the carry; round trip sum_j d_j 2^(Mj) = a_i and the digit ranges;
* NTT mod p: a radix-2 decimation-in-frequency transform against the naive
  O(n^2) DFT, and inverse after forward = n times the identity;
* the two convolutions (§2.1): C^- = AB mod (x^K - 1) by a length-K cyclic
  DFT convolution and C^+ = AB mod (x^K + 1) by the twisted one
  (x -> theta x, theta a primitive 2K-th root), against schoolbook
  reduction mod x^K -+ 1;
* recovery (§2.2, reading R9): c_{i,j} = (c^-_{i,j} + c^+_{i,j})/2 and
  c_{i,j+K} = (c^-_{i,j} - c^+_{i,j})/2 are exact integers and
  c_i = sum_{j<2K} c_{i,j} 2^(Mj);
* CRT (§4, readings R3 and R6): Garner's mixed radix against the direct
  centred lift, with m > 4H for H = min(na, nb) K 2^(2M-2);
* the whole method on small random polynomials against Python's own
  product, for several (K, M) splits.

The model uses its own primes (998244353 = 119 2^23 + 1, 469762049 =
7 2^26 + 1, 167772161 = 5 2^25 + 1, all with primitive root 3) and its own
arithmetic; it shares nothing with the CUDA library or the C oracle.
"""
import math

import numpy as np
import pytest

from bigint_util import brute_product

PRIMES = [998244353, 469762049, 167772161]
GEN = 3


def root(p, n, inverse=False):
    """Primitive n-th root of unity mod p (n | p - 1)."""
    w = pow(GEN, (p - 1) // n, p)
    return pow(w, p - 2, p) if inverse else w


# ---- split -------------------------------------------------------------------

def split(a, K, M):
    """Balanced digits of a (|a| < 2^(N-1), N = KM) per reading R1."""
    N = K * M
    u = a % (1 << N)  # N-bit two's complement
    fields = [(u >> (M * j)) & ((1 << M) - 1) for j in range(K)]
    half = 1 << (M - 1)
    d, carry = [], 0
    for j in range(K - 1):
        t = fields[j] + carry
        if t >= half:
            d.append(t - (1 << M))
            carry = 1
        else:
            d.append(t)
            carry = 0
    top = fields[K - 1]
    top = top - (1 << M) if top >= half else top
    d.append(top + carry)
    return d


@pytest.mark.parametrize("K,M", [(2, 3), (4, 5), (8, 8), (16, 33), (2, 62)])
def test_split_round_trip_and_ranges(K, M):
    N = K * M
    rng = np.random.default_rng(K * 100 + M)
    vals = [0, 1, -1, (1 << (N - 1)) - 1, -(1 << (N - 1)) + 1, -(1 << (N - 1))]
    vals += [int.from_bytes(rng.bytes(N // 8 + 1), "little") % (1 << (N - 1)) * (1 if rng.random() < .5 else -1)
             for _ in range(50)]
    half = 1 << (M - 1)
    for a in vals:
        d = split(a, K, M)
        assert sum(x << (M * j) for j, x in enumerate(d)) == a
        assert all(-half <= x <= half - 1 for x in d[:-1])
        assert -half <= d[-1] <= half


def test_paper_digit_range_cannot_cover_every_coefficient():
    """With every digit in [-2^(M-1), 2^(M-1) - 1] (§2) the largest value is
    sum_j (2^(M-1) - 1) 2^(Mj) < 2^(N-1) - 1, so the top digit must be
    allowed 2^(M-1) (reading R1)."""
    K, M = 2, 2
    top = sum(((1 << (M - 1)) - 1) << (M * j) for j in range(K))
    assert top < (1 << (K * M - 1)) - 1
    d = split((1 << (K * M - 1)) - 1, K, M)
    assert d[-1] == 1 << (M - 1)


# ---- NTT -----------------------------------------------------------------------

def dft_naive(x, p, w):
    n = len(x)
    return [sum(x[k] * pow(w, j * k, p) for k in range(n)) % p for j in range(n)]


def ntt_dif(x, p, w):
    """Radix-2 decimation in frequency, natural order in, natural order out
    (the bit-reversal undone at the end)."""
    x = list(x)
    n = len(x)
    h = n // 2
    while h >= 1:
        wh = pow(w, n // (2 * h), p)
        for b in range(0, n, 2 * h):
            t = 1
            for k in range(h):
                u, v = x[b + k], x[b + k + h]
                x[b + k] = (u + v) % p
                x[b + k + h] = (u - v) * t % p
                t = t * wh % p
        h //= 2
    bits = n.bit_length() - 1
    return [x[int(format(j, "0%db" % bits)[::-1], 2) if bits else 0] for j in range(n)]


@pytest.mark.parametrize("n", [1, 2, 4, 16, 64, 256])
@pytest.mark.parametrize("p", PRIMES)
def test_ntt_matches_naive_dft_and_inverts(n, p):
    rng = np.random.default_rng(n)
    x = [int(v) % p for v in rng.integers(0, 2**62, n)]
    w = root(p, n)
    X = ntt_dif(x, p, w)
    assert X == dft_naive(x, p, w)
    back = ntt_dif(X, p, root(p, n, inverse=True))
    assert [v * pow(n, p - 2, p) % p for v in back] == x


# ---- the two convolutions ------------------------------------------------------

def schoolbook_mod(a, b, K, sign, p):
    """a*b mod (x^K - sign) over Z/p."""
    c = [0] * K
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            k = i + j
            if k >= K:
                c[k - K] += sign * x * y
            else:
                c[k] += x * y
    return [v % p for v in c]


def cyclic(a, b, p):
    K = len(a)
    w = root(p, K)
    C = [x * y % p for x, y in zip(ntt_dif(a, p, w), ntt_dif(b, p, w))]
    return [v * pow(K, p - 2, p) % p for v in ntt_dif(C, p, root(p, K, True))]


def negacyclic(a, b, p):
    """Twist x -> theta x (theta a primitive 2K-th root), cyclic, untwist."""
    K = len(a)
    th = root(p, 2 * K)
    at = [x * pow(th, j, p) % p for j, x in enumerate(a)]
    bt = [x * pow(th, j, p) % p for j, x in enumerate(b)]
    c = cyclic(at, bt, p)
    thi = pow(th, p - 2, p)
    return [x * pow(thi, j, p) % p for j, x in enumerate(c)]


@pytest.mark.parametrize("K", [1, 2, 8, 32])
def test_cyclic_and_negacyclic_convolutions(K):
    p = PRIMES[0]
    rng = np.random.default_rng(K)
    a = [int(v) for v in rng.integers(0, p, K)]
    b = [int(v) for v in rng.integers(0, p, K)]
    assert cyclic(a, b, p) == schoolbook_mod(a, b, K, +1, p)
    assert negacyclic(a, b, p) == schoolbook_mod(a, b, K, -1, p)


# ---- CRT -------------------------------------------------------------------------

def garner(res, primes):
    """Mixed-radix digits v_t, then X = v0 + p0 (v1 + p1 (v2 + ...))."""
    v = []
    for t, (r, p) in enumerate(zip(res, primes)):
        y = r
        for s in range(t):
            y = (y - v[s]) * pow(primes[s], p - 2, p) % p
        v.append(y)
    X = 0
    for t in reversed(range(len(primes))):
        X = X * primes[t] + v[t]
    return X


def centred(X, m):
    return X - m if 2 * X > m else X  # m odd: no tie (reading R6)


def test_garner_matches_centred_lift():
    m = math.prod(PRIMES)
    rng = np.random.default_rng(7)
    for _ in range(200):
        c = int.from_bytes(rng.bytes(11), "little") % m - m // 2
        res = [c % p for p in PRIMES]
        assert centred(garner(res, PRIMES), m) == c


# ---- the whole method -------------------------------------------------------------

def method_product(a, b, K, M, primes):
    """§2-§2.2 with the CRT of §4: split, both convolutions per prime with a
    zero-padded y convolution, per-digit halving, CRT, recombination."""
    na, nb = len(a), len(b)
    nc = na + nb - 1
    A = [split(x, K, M) for x in a]
    B = [split(x, K, M) for x in b]
    H = min(na, nb) * K * (1 << (2 * M - 2))
    m = math.prod(primes)
    assert m > 4 * H, "not enough primes for the bound (reading R3)"
    digits = [[None] * (2 * K) for _ in range(nc)]
    per_prime = []
    for p in primes:
        # c^-_{i,j} and c^+_{i,j} mod p: y convolution by schoolbook (the y
        # transform is the same DFT machinery as x), x by the two DFT convolutions
        cm = [[0] * K for _ in range(nc)]
        cp = [[0] * K for _ in range(nc)]
        for i in range(na):
            for j in range(nb):
                ai = [x % p for x in A[i]]
                bj = [x % p for x in B[j]]
                cyc = cyclic(ai, bj, p)
                neg = negacyclic(ai, bj, p)
                for k in range(K):
                    cm[i + j][k] = (cm[i + j][k] + cyc[k]) % p
                    cp[i + j][k] = (cp[i + j][k] + neg[k]) % p
        inv2 = pow(2, p - 2, p)
        lo = [[(cm[i][k] + cp[i][k]) * inv2 % p for k in range(K)] for i in range(nc)]
        hi = [[(cm[i][k] - cp[i][k]) * inv2 % p for k in range(K)] for i in range(nc)]
        per_prime.append((lo, hi))
    for i in range(nc):
        for k in range(K):
            digits[i][k] = centred(garner([pp[0][i][k] for pp in per_prime], primes), m)
            digits[i][k + K] = centred(garner([pp[1][i][k] for pp in per_prime], primes), m)
            assert abs(digits[i][k]) <= H and abs(digits[i][k + K]) <= H
    return [sum(d << (M * j) for j, d in enumerate(row)) for row in digits]


@pytest.mark.parametrize("na,nb,bits,K,M,r", [(1, 1, 5, 2, 3, 1), (3, 2, 7, 2, 4, 2), (4, 4, 20, 4, 6, 2),
                                               (5, 3, 30, 8, 4, 2), (6, 6, 60, 4, 16, 3), (2, 7, 40, 8, 6, 2)])
def test_method_model_equals_plain_product(na, nb, bits, K, M, r):
    assert K * M >= bits + 1
    rng = np.random.default_rng(na + nb + bits)

    def rand():
        v = int.from_bytes(rng.bytes(bits // 8 + 1), "little") % (1 << bits)
        return -v if rng.random() < 0.5 else v

    a = [rand() for _ in range(na)]
    b = [rand() for _ in range(nb)]
    assert method_product(a, b, K, M, PRIMES[:r]) == brute_product(a, b)


def test_method_model_extreme_digits():
    """Every balanced digit -2^(M-1): the digit products reach the bound H."""
    K, M = 4, 5
    v = sum((-(1 << (M - 1))) << (M * j) for j in range(K - 1))
    a, b = [v] * 3, [v] * 3
    assert method_product(a, b, K, M, PRIMES[:2]) == brute_product(a, b)
