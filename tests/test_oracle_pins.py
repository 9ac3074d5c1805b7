"""Pins for the CPU oracle (-m "not gpu").

The oracle computes c = a*b from its definition (§1: c(y) = a(y) b(y) over
Z).  Before it is trusted, it is checked here against things other than
itself: Python's independent integers (brute force and Kronecker
substitution), the closed form for constant polynomials, the exact
identities C(1) = A(1)B(1) and C(-1) = A(-1)B(-1), and evaluation modulo
independent 61-bit primes.  The mutation tests plant known mistakes in the
oracle and show that at least one pin fails for each.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from bigint_util import (CHECK_PRIMES, brute_product, eval_at, eval_mod_py, from_ints,
                         kronecker_product, terms, to_ints)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lc(na, nb, ba, bb):
    return W.Product(na, nb, ba, bb).lc


def test_check_primes_are_prime():
    sympy = pytest.importorskip("sympy")
    for q in CHECK_PRIMES:
        assert sympy.isprime(q)


@pytest.mark.parametrize("na,nb,ba,bb", [
    (1, 1, 1, 1), (1, 5, 32, 7), (3, 2, 33, 64), (7, 7, 100, 100), (4, 9, 31, 200),
    (16, 3, 255, 1), (2, 2, 4096, 4096), (12, 12, 64, 96)])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_python_int(na, nb, ba, bb, seed):
    """Tiny random inputs: oracle == double loop over Python ints."""
    rng = np.random.default_rng(1000 + seed)
    a = W.random_poly(rng, na, ba)
    b = W.random_poly(rng, nb, bb)
    lc = _lc(na, nb, ba, bb)
    c = oracle.polymul(a, b, lc, threads=2)
    want = brute_product(to_ints(*a), to_ints(*b))
    assert to_ints(*c) == want
    # zero is always +0
    assert all(s == 0 for v, s in zip(want, c[1]) if v == 0)


def test_signs_and_zero_normalisation():
    a = from_ints([0, -1, 5, 0], 1)
    b = from_ints([-3, 0, 0], 1)
    c = oracle.polymul(a, b, 3, threads=1)
    assert to_ints(*c) == brute_product([0, -1, 5, 0], [-3, 0, 0])
    # c_0 = 0*(-3) = 0 -> stored as +0; c_1 = 3
    assert c[1][0] == 0 and to_ints(*c)[1] == 3


def test_cancellation_to_zero():
    # (1 + y)(1 - y) = 1 - y^2 : middle coefficient cancels exactly
    a = from_ints([1, 1], 1)
    b = from_ints([1, -1], 1)
    c = oracle.polymul(a, b, 1)
    assert to_ints(*c) == [1, 0, -1]
    assert list(c[1]) == [0, 0, 1]


@pytest.mark.parametrize("na,nb,bits", [(200, 200, 300), (333, 57, 1000), (64, 513, 96)])
def test_kronecker_mid_size(na, nb, bits):
    """Mid sizes: schoolbook oracle == one big-integer product (Kronecker)."""
    rng = np.random.default_rng(7 + na)
    a = W.random_poly(rng, na, bits)
    b = W.random_poly(rng, nb, bits)
    lc = _lc(na, nb, bits, bits)
    c = oracle.polymul(a, b, lc)
    want = kronecker_product(to_ints(*a), to_ints(*b), 32 * lc + 2)
    assert to_ints(*c) == want


@pytest.mark.parametrize("na,nb,bits,negative", [(64, 64, 4096, False), (50, 17, 300, True),
                                                 (1, 9, 33, False), (33, 1, 64, True)])
def test_closed_form_constant(na, nb, bits, negative):
    """All coefficients alpha=+-(2^bits-1): c_k = terms(k) * alpha_a * alpha_b."""
    a = W.constant_poly(na, bits, negative=negative)
    b = W.constant_poly(nb, bits)
    alpha = (1 << bits) - 1
    lc = _lc(na, nb, bits, bits)
    c = oracle.polymul(a, b, lc)
    sa = -1 if negative else 1
    want = [sa * terms(k, na, nb) * alpha * alpha for k in range(na + nb - 1)]
    assert to_ints(*c) == want


@pytest.mark.parametrize("seed", [0, 1])
def test_identities_at_plus_minus_one(seed):
    _, a, b = W.small_dense(seed=seed, n=300, bits=255)
    lc = _lc(300, 300, 255, 255)
    c = oracle.polymul(a, b, lc)
    A, B, C = to_ints(*a), to_ints(*b), to_ints(*c)
    for t in (1, -1, 2):
        assert eval_at(C, t) == eval_at(A, t) * eval_at(B, t)


def test_eval_mod_matches_python():
    rng = np.random.default_rng(5)
    a = W.random_poly(rng, 40, 200)
    vals = to_ints(*a)
    for q in CHECK_PRIMES:
        for t in (0, 1, 2, 12345678901234567, q - 1):
            assert oracle.eval_mod(a, t, q) == eval_mod_py(vals, t, q)


def test_eval_mod_product_identity():
    _, a, b = W.small_dense(seed=3, n=500, bits=255)
    c = oracle.polymul(a, b, _lc(500, 500, 255, 255))
    rng = np.random.default_rng(9)
    for q in CHECK_PRIMES:
        t = int(rng.integers(2, 2**60))
        assert oracle.eval_mod(c, t, q) == oracle.eval_mod(a, t, q) * oracle.eval_mod(b, t, q) % q


def test_coeffs_matches_full():
    _, a, b = W.small_dense(seed=4, n=130, bits=90)
    lc = _lc(130, 130, 90, 90)
    c = oracle.polymul(a, b, lc)
    ks = [0, 1, 64, 129, 200, 258]
    s = oracle.coeffs(ks, a, b, lc, threads=3)
    assert np.array_equal(s[0], c[0][ks]) and np.array_equal(s[1], c[1][ks])


def test_thread_count_invariance():
    _, a, b = W.small_dense(seed=6, n=257, bits=64)
    lc = _lc(257, 257, 64, 64)
    c1 = oracle.polymul(a, b, lc, threads=1)
    c7 = oracle.polymul(a, b, lc, threads=7)
    assert np.array_equal(c1[0], c7[0]) and np.array_equal(c1[1], c7[1])


def test_too_small_output_is_an_error():
    a = W.constant_poly(4, 64)
    with pytest.raises(RuntimeError):
        oracle.polymul(a, a, 1)


# ---- planted mistakes: each must be caught by at least one pin ------------

def _pins_fail(a, b, c, lc) -> list[str]:
    """Return the names of the pins that reject output c for inputs a, b."""
    A, B, C = to_ints(*a), to_ints(*b), to_ints(*c)
    failed = []
    if C != brute_product(A, B):
        failed.append("brute")
    if eval_at(C, 1) != eval_at(A, 1) * eval_at(B, 1):
        failed.append("C(1)")
    if eval_at(C, -1) != eval_at(A, -1) * eval_at(B, -1):
        failed.append("C(-1)")
    for q in CHECK_PRIMES[:1]:
        t = 987654321987
        if oracle.eval_mod(c, t, q) != oracle.eval_mod(a, t, q) * oracle.eval_mod(b, t, q) % q:
            failed.append("mod")
    return failed


@pytest.mark.parametrize("mutation,name", [(1, "dropped term"), (2, "dropped sign of b"),
                                           (3, "off-by-one index"), (4, "lost limb carry"),
                                           (5, "limbs read big-endian")])
def test_planted_mistakes_are_caught(mutation, name):
    rng = np.random.default_rng(77)
    a = W.random_poly(rng, 9, 96)
    b = W.random_poly(rng, 7, 96)
    lc = _lc(9, 7, 96, 96)
    good = oracle.polymul(a, b, lc)
    assert _pins_fail(a, b, good, lc) == []
    bad = oracle.polymul(a, b, lc, mutation=mutation)
    failed = _pins_fail(a, b, bad, lc)
    # the whole-output identities alone (no brute force) must also catch it
    assert failed and any(f in failed for f in ("C(1)", "C(-1)", "mod")), (name, failed)


# ---- stored values (written by tests/golden/make_golden.py from oracle/ only)

def test_golden_small_dense_digest():
    with open(os.path.join(GOLDEN, "small_dense_seed0.json")) as f:
        g = json.load(f)
    sh, a, b = W.small_dense(seed=0)
    c = oracle.polymul(a, b, sh.lc)
    h = hashlib.sha256(c[0].tobytes() + c[1].tobytes()).hexdigest()
    assert h == g["sha256"]
    # Input digest too, so a change of the generator is noticed separately.
    hin = hashlib.sha256(a[0].tobytes() + a[1].tobytes() + b[0].tobytes() + b[1].tobytes()).hexdigest()
    assert hin == g["inputs_sha256"]


def test_golden_hand_worked_examples():
    """Small products worked by hand (tests/golden/hand_examples.json)."""
    with open(os.path.join(GOLDEN, "hand_examples.json")) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        A = [int(x) for x in case["a"]]
        B = [int(x) for x in case["b"]]
        C = [int(x) for x in case["c"]]
        ba = max(1, max(abs(x) for x in A).bit_length())
        bb = max(1, max(abs(x) for x in B).bit_length())
        la, lb = W.limbs_for_bits(ba), W.limbs_for_bits(bb)
        lc = W.Product(len(A), len(B), ba, bb).lc
        c = oracle.polymul(from_ints(A, la), from_ints(B, lb), lc)
        assert to_ints(*c) == C, case["why"]


def test_small_dense_full_size_kronecker():
    """The whole small dense product (1024 x 1024 coefficients, 255 bits)
    equals one Kronecker-substituted big-integer product done by Python."""
    sh, a, b = W.small_dense(seed=0)
    c = oracle.polymul(a, b, sh.lc)
    want = kronecker_product(to_ints(*a), to_ints(*b), 32 * sh.lc + 2)
    assert to_ints(*c) == want


# ---------------------------------------------------------------------------
# The full-output oracle at large sizes: Kronecker substitution with the
# oracle's own Karatsuba (oracle.polymul_kron).  Pinned to Python's
# independent integers (the integer product alone, across the schoolbook
# threshold, odd and uneven splits, carries through all-ones limbs) and to
# the schoolbook definition on whole outputs (signs, zeros, unbalanced
# degrees, extreme magnitudes, cancellation).
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("limbs", [1, 2, 63, 64, 65, 127, 129, 300, 1001, 4096])
@pytest.mark.parametrize("threads", [1, 5])
def test_karatsuba_matches_python_integers(limbs, threads):
    rng = np.random.default_rng(limbs * 7 + threads)
    for kind in ("random", "ones", "lopsided"):
        if kind == "random":
            x = int.from_bytes(rng.bytes(4 * limbs), "little")
            y = int.from_bytes(rng.bytes(4 * limbs), "little")
        elif kind == "ones":
            x = y = (1 << (32 * limbs)) - 1
        else:  # one operand much shorter: the upper halves are zero
            x = int.from_bytes(rng.bytes(4 * limbs), "little")
            y = int.from_bytes(rng.bytes(4), "little") | 1
        assert oracle.kara_mul(x, y, threads=threads) == x * y


@pytest.mark.parametrize("na,nb,ba,bb", [
    (1, 1, 1, 1), (2, 1, 4096, 5), (5, 3, 70, 33), (64, 64, 1, 1), (300, 257, 255, 255),
    (1024, 1024, 255, 255), (700, 1500, 1000, 64), (3, 2000, 2048, 32), (129, 128, 4096, 4096)])
def test_kronecker_karatsuba_matches_schoolbook(na, nb, ba, bb):
    rng = np.random.default_rng(na * 31 + nb)
    a = W.random_poly(rng, na, ba)
    b = W.random_poly(rng, nb, bb)
    lc = _lc(na, nb, ba, bb)
    want = oracle.polymul(a, b, lc)
    got = oracle.polymul_kron(a, b, lc, threads=3)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_kronecker_karatsuba_extremes_and_cancellation():
    # every magnitude 2^bits - 1 with all signs equal: the largest |c_k|
    for neg in (False, True):
        a = W.constant_poly(500, 300, negative=neg)
        b = W.constant_poly(400, 300)
        lc = _lc(500, 400, 300, 300)
        want = oracle.polymul(a, b, lc)
        got = oracle.polymul_kron(a, b, lc)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    # (y - 1)(y + 1) = y^2 - 1 with huge equal magnitudes: c_1 cancels to +0
    big = (1 << 2000) - 12345
    a = from_ints([-big, big], 63)
    b = from_ints([big, big], 63)
    got = oracle.polymul_kron(a, b, _lc(2, 2, 2016, 2016))
    assert to_ints(*got) == [-big * big, 0, big * big] and got[1][1] == 0
    # zero polynomials
    z = from_ints([0] * 17, 4)
    got = oracle.polymul_kron(z, W.random_poly(np.random.default_rng(3), 9, 100), _lc(17, 9, 128, 100))
    assert not got[0].any() and not got[1].any()


def test_kronecker_karatsuba_rejects_a_too_small_output():
    a = W.constant_poly(64, 256)
    with pytest.raises(RuntimeError):
        oracle.polymul_kron(a, a, 8)  # |c_k| needs 17 limbs


def test_full_size_digests_were_written_by_the_oracle():
    """The stored full-size digests (tests/golden/make_full_digests.py) name
    the same seeded inputs the workloads module generates today."""
    path = os.path.join(GOLDEN, "full_size_digests.json")
    if not os.path.exists(path):
        pytest.skip("no full-size digests")
    store = json.load(open(path))
    makers = {"large_dense": lambda: W.large_dense(seed=1), "huge_dense": lambda: W.huge_dense(seed=2),
              "huge_mixed": lambda: W.huge_mixed(seed=2)}
    for name, rec in store.items():
        sh, a, b = makers[name]()
        assert rec["nc"] == sh.nc and rec["lc"] == sh.lc
        assert rec["inputs_sha256"] == hashlib.sha256(a[0].tobytes() + a[1].tobytes() + b[0].tobytes() +
                                                      b[1].tobytes()).hexdigest()
        assert "oracle.polymul_kron" in rec["written_by"]
