"""Test-side big-integer helpers built on Python's own ``int``.

Python's arbitrary-precision integers are an implementation independent of
both the C oracle and the CUDA library, so conversions and checks written
with them can pin either side.
"""
from __future__ import annotations

import numpy as np


def to_ints(limbs: np.ndarray, neg: np.ndarray) -> list[int]:
    """Sign-magnitude limb rows -> list of Python ints."""
    limbs = np.ascontiguousarray(limbs, dtype="<u4")
    out = []
    for row, s in zip(limbs, neg):
        v = int.from_bytes(row.tobytes(), "little")
        out.append(-v if s else v)
    return out


def from_ints(vals, L: int):
    """List of Python ints -> (limbs (n, L) uint32, neg uint8); raises if one does not fit."""
    n = len(vals)
    limbs = np.zeros((n, L), dtype="<u4")
    neg = np.zeros(n, dtype=np.uint8)
    for i, v in enumerate(vals):
        m = -v if v < 0 else v
        if m >= 1 << (32 * L):
            raise OverflowError("value does not fit in %d limbs" % L)
        limbs[i] = np.frombuffer(m.to_bytes(4 * L, "little"), dtype="<u4")
        neg[i] = 1 if v < 0 else 0
    return limbs.astype(np.uint32), neg


def brute_product(a: list[int], b: list[int]) -> list[int]:
    """c_k = sum_{i+j=k} a_i b_j with Python ints (tiny inputs only)."""
    c = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            c[i + j] += x * y
    return c


def kronecker_product(a: list[int], b: list[int], slot_bits: int) -> list[int]:
    """Product through Kronecker substitution: one big integer product.

    a(2^s) and b(2^s) are formed as single Python integers with signed slots
    of s bits, multiplied once, and c is read back slot by slot with a
    borrow.  Requires 2*max|c_k| < 2^s.
    """
    s = slot_bits
    A = sum(x << (s * i) for i, x in enumerate(a))
    B = sum(y << (s * j) for j, y in enumerate(b))
    C = A * B
    out = []
    half = 1 << (s - 1)
    mask = (1 << s) - 1
    for _ in range(len(a) + len(b) - 1):
        r = C & mask
        if r >= half:
            r -= 1 << s
        out.append(r)
        C = (C - r) >> s
    if C != 0:
        raise ValueError("slot width too small")
    return out


def eval_at(vals: list[int], t: int) -> int:
    """Exact evaluation at an integer point (Horner)."""
    acc = 0
    for v in reversed(vals):
        acc = acc * t + v
    return acc


def eval_mod_py(vals: list[int], t: int, q: int) -> int:
    acc = 0
    for v in reversed(vals):
        acc = (acc * t + v) % q
    return acc


def terms(k: int, na: int, nb: int) -> int:
    """Number of pairs (i, j) with i + j = k, 0 <= i < na, 0 <= j < nb."""
    lo = max(0, k - (nb - 1))
    hi = min(k, na - 1)
    return max(0, hi - lo + 1)


# Independent 61-bit primes (none is an NTT prime of the library: those are
# below 2^30) for Schwartz-Zippel checks of whole outputs.
CHECK_PRIMES = [(1 << 61) - 1, 2305843009213693921, 2305843009213693907]


GOLDEN_DIR = __import__("os").path.join(__import__("os").path.dirname(__import__("os").path.abspath(__file__)),
                                        "golden")


def full_output_digest(c, cn):
    """SHA-256 of a whole product as tests/golden/make_full_digests.py
    writes it: little-endian uint32 limb rows, then the sign bytes."""
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(c).astype("<u4").tobytes() +
                          np.ascontiguousarray(cn).tobytes()).hexdigest()


def stored_full_digest(name):
    """The oracle's full-size digest of workload `name`
    (tests/golden/full_size_digests.json), or None."""
    import json
    import os
    path = os.path.join(GOLDEN_DIR, "full_size_digests.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(name)
    return rec["sha256"] if rec else None
