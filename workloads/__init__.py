"""Seeded synthetic inputs for dense Z[y] products (§4: random dense a, b).

This module is shared by the CPU oracle side (tests, the oracle baseline in
``bench.py``) and the CUDA side.  It draws random numbers and lays them out in
the library's operand format; it holds none of the multiplication method's
arithmetic (no splitting, transforms, residues or recombination).

Operand format (sign-magnitude, 32-bit little-endian limbs):
  limbs : uint32 array of shape (n, L), L = ceil(bits / 32); row i is |a_i|
  neg   : uint8 array of shape (n,), 1 where a_i < 0 (never set for a_i = 0)
  |a_i| < 2**bits for every i.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def limbs_for_bits(bits: int) -> int:
    """Number of 32-bit limbs that hold a magnitude below 2**bits."""
    if bits < 1:
        raise ValueError("bits must be >= 1")
    return (bits + 31) // 32


def random_poly(rng: np.random.Generator, n: int, bits: int, *, signed: bool = True,
                row_bits: np.ndarray | None = None, stride_bits: int | None = None):
    """Random dense polynomial with n coefficients and |a_i| < 2**bits.

    Magnitudes are the low ``bits`` bits of uniform random words (so they are
    uniform in [0, 2**bits)); the sign is an independent fair coin and a zero
    magnitude is always stored as +0.

    ``row_bits`` (optional, shape (n,)) gives a per-coefficient bit bound
    <= bits, for the mixed-size workloads; ``stride_bits`` (>= bits) widens
    the limb stride beyond what ``bits`` needs.
    """
    L = limbs_for_bits(stride_bits if stride_bits is not None else bits)
    limbs = rng.integers(0, 2**32, size=(n, L), dtype=np.uint64).astype(np.uint32)
    rb = np.full(n, bits, dtype=np.int64) if row_bits is None else np.asarray(row_bits, np.int64)
    if np.any(rb > bits) or np.any(rb < 1):
        raise ValueError("row_bits must lie in [1, bits]")
    # Mask every row to its own bit bound.
    col = np.arange(L, dtype=np.int64)[None, :]
    full = rb[:, None] // 32
    rem = rb[:, None] % 32
    keep_all = col < full
    partial = (col == full) & (rem > 0)
    mask = np.where(keep_all, np.uint64(0xFFFFFFFF),
                    np.where(partial, (np.uint64(1) << rem.astype(np.uint64)) - np.uint64(1),
                             np.uint64(0))).astype(np.uint32)
    limbs &= mask
    if signed:
        neg = rng.integers(0, 2, size=n, dtype=np.uint8)
    else:
        neg = np.zeros(n, dtype=np.uint8)
    neg[~limbs.any(axis=1)] = 0
    return np.ascontiguousarray(limbs), np.ascontiguousarray(neg)


def constant_poly(n: int, bits: int, value_bits: int | None = None, negative: bool = False):
    """Every coefficient equal to +-(2**value_bits - 1) (default value_bits = bits)."""
    vb = bits if value_bits is None else value_bits
    L = limbs_for_bits(bits)
    limbs = np.zeros((n, L), dtype=np.uint32)
    full, rem = divmod(vb, 32)
    limbs[:, :full] = 0xFFFFFFFF
    if rem:
        limbs[:, full] = (1 << rem) - 1
    neg = np.full(n, 1 if negative else 0, dtype=np.uint8)
    if vb == 0:
        neg[:] = 0
    return limbs, neg


@dataclass(frozen=True)
class Product:
    """One product a*b: numbers of coefficients and magnitude bit bounds."""
    na: int
    nb: int
    bits_a: int
    bits_b: int

    @property
    def nc(self) -> int:
        return self.na + self.nb - 1

    @property
    def la(self) -> int:
        return limbs_for_bits(self.bits_a)

    @property
    def lb(self) -> int:
        return limbs_for_bits(self.bits_b)

    @property
    def lc(self) -> int:
        """Output limb stride: |c_k| < min(na, nb) * 2**(bits_a + bits_b)."""
        m = min(self.na, self.nb)
        lg = 0 if m <= 1 else math.ceil(math.log2(m))
        return (self.bits_a + self.bits_b + lg + 31) // 32


# ---------------------------------------------------------------------------
# The five workload families (degree d-1 means d coefficients).
# ---------------------------------------------------------------------------

def small_dense(seed: int = 0, n: int = 1024, bits: int = 255):
    """Two degree-1023 polynomials, |coefficients| < 2**255, seed 0."""
    rng = np.random.default_rng(seed)
    a = random_poly(rng, n, bits)
    b = random_poly(rng, n, bits)
    return Product(n, n, bits, bits), a, b


def large_dense(seed: int = 1, n: int = 32768, bits: int = 4096):
    """Two degree-32767 polynomials, |coefficients| < 2**4096, seed 1."""
    rng = np.random.default_rng(seed)
    a = random_poly(rng, n, bits)
    b = random_poly(rng, n, bits)
    return Product(n, n, bits, bits), a, b


def large_all_ones(n: int = 32768, bits: int = 4096):
    """Every coefficient of a and b equal to 2**bits - 1 (long carry runs)."""
    a = constant_poly(n, bits)
    b = constant_poly(n, bits)
    return Product(n, n, bits, bits), a, b


def huge_dense(seed: int = 2, n: int = 262144, bits: int = 1024):
    """Two degree-262143 polynomials, |coefficients| < 2**1024, seed 2."""
    rng = np.random.default_rng(seed)
    a = random_poly(rng, n, bits)
    b = random_poly(rng, n, bits)
    return Product(n, n, bits, bits), a, b


def huge_mixed(seed: int = 2, n: int = 262144, small_bits: int = 64, big_bits: int = 2048):
    """Half of the positions < 2**64, the rest < 2**2048 (random positions)."""
    rng = np.random.default_rng(seed + 1000)
    out = []
    for _ in range(2):
        rb = np.where(rng.integers(0, 2, size=n) == 0, small_bits, big_bits)
        out.append(random_poly(rng, n, big_bits, row_bits=rb))
    return Product(n, n, big_bits, big_bits), out[0], out[1]


def taylor_dense(seed: int = 5, n: int = 16384, bits: int = 4096):
    """Taylor-shift input: n random signed coefficients below 2^bits
    (the shape of the root-isolation use in §1: dense, large coefficients)."""
    rng = np.random.default_rng(seed)
    return (n, bits), random_poly(rng, n, bits)


def batch_shapes(seed: int = 3, count: int = 4096, dmin: int = 16, dmax: int = 8192,
                 bmin: int = 32, bmax: int = 4096):
    """Shapes for the batched workload: log-uniform degrees and bit bounds."""
    rng = np.random.default_rng(seed)
    u = rng.random((count, 4))
    na = np.floor(np.exp(np.log(dmin) + u[:, 0] * (np.log(dmax) - np.log(dmin)))).astype(np.int64)
    nb = np.floor(np.exp(np.log(dmin) + u[:, 1] * (np.log(dmax) - np.log(dmin)))).astype(np.int64)
    ba = np.floor(np.exp(np.log(bmin) + u[:, 2] * (np.log(bmax) - np.log(bmin)))).astype(np.int64)
    bb = np.floor(np.exp(np.log(bmin) + u[:, 3] * (np.log(bmax) - np.log(bmin)))).astype(np.int64)
    return [Product(int(x), int(y), int(p), int(q)) for x, y, p, q in zip(na, nb, ba, bb)]


def batch_operands(shapes, seed: int = 3):
    """Random operands for a list of Product shapes (independent stream per item)."""
    ss = np.random.SeedSequence(seed)
    out = []
    for sh, child in zip(shapes, ss.spawn(len(shapes))):
        rng = np.random.default_rng(child)
        out.append((random_poly(rng, sh.na, sh.bits_a), random_poly(rng, sh.nb, sh.bits_b)))
    return out


def sweep_grid(dmin_log: int = 6, dmax_log: int = 20, bmin_log: int = 5, bmax_log: int = 14):
    """The (degree, bits) grid of the dispatch sweep: powers of two on both axes."""
    return [(1 << dl, 1 << bl) for dl in range(dmin_log, dmax_log + 1)
            for bl in range(bmin_log, bmax_log + 1)]


def sweep_unbalanced(seed: int = 4, count: int = 60):
    """Unbalanced shapes added to the dispatch sweep: (na, nb, bits_a,
    bits_b) drawn like the batched workload (log-uniform degrees in
    [16, 65536], bit bounds in [16, 4096]), from the sweep's seed."""
    shapes = batch_shapes(seed=seed, count=count, dmin=16, dmax=65536, bmin=16, bmax=4096)
    return [(s.na, s.nb, s.bits_a, s.bits_b) for s in shapes]
