"""The arithmetic identities two GPU kernels rely on, restated with Python
integers and checked exhaustively or on random values -- so the reasoning
behind them is pinned on the CPU (the kernels themselves are compared with
the oracle by the GPU tests).

Randomised product check (csrc/ipm_validate.cu), q = 2^61 - 1:
* a limb x < 2^32 times 2^e (e < 61) modulo q is the rotation
  ((x << e) mod 2^64 & q) | (x >> (61 - e)) of the 64-bit kernel code;
* 2^(32 l) mod q = 2^(32 l mod 61), and 32 (l + 32) = 32 l + 48 mod 61, the
  lane stride of the limb loop;
* eight rotated limbs (each < 2^61) sum below 2^64, so one reduction per
  eight suffices.

Tensor-core radix-16 stage (ntt_stages.cuh, stage_tc16), for a prime p:
* with x_k = sum_s x_k^(s) 2^(8s) (bytes) and C[j][k][s] = E[j][k] 2^(8s)
  2^32 mod p split into bytes C^(l), V_j = sum_l 2^(8l) D_l[j] with
  D_l[j] = sum_{k,s} C^(l)[j][k][s] x_k^(s) is congruent to 2^32 sum_k
  E[j][k] x_k, every D_l < 2^22 and V < 2^46 < p 2^32; Montgomery's REDC of
  V gives the DFT output in [0, 2p).
"""
import numpy as np
import pytest

Q = (1 << 61) - 1
MASK64 = (1 << 64) - 1


def rot61(x, e):
    if e == 0:
        return x
    return (((x << e) & MASK64) & Q) | (x >> (61 - e))


def test_rotation_is_multiplication_by_a_power_of_two():
    rng = np.random.default_rng(1)
    xs = [0, 1, 0xFFFFFFFF, 0x80000000] + [int(v) for v in rng.integers(0, 2**32, 200)]
    for e in range(61):
        for x in xs:
            assert rot61(x, e) == (x << e) % Q


def test_limb_weights_and_lane_stride():
    for lane in range(32):
        e = (32 * lane) % 61
        for k in range(20):
            l = lane + 32 * k
            assert pow(2, 32 * l, Q) == pow(2, e, Q) == 1 << e
            e = (e + 48) % 61


def test_eight_rotated_limbs_fit_64_bits():
    assert 8 * (Q - 1) < 1 << 64  # rot61 of a value below 2^61 stays below 2^61
    assert all(rot61(0xFFFFFFFF, e) < 1 << 61 for e in range(61))


def brev4(j):
    return int(format(j, "04b")[::-1], 2)


@pytest.mark.parametrize("p", [1012924417, 1004535809, 998244353])
@pytest.mark.parametrize("forward", [True, False])
def test_byte_slice_dft_identity(p, forward):
    # a primitive 16th root (any; the identity does not depend on which)
    w = None
    for cand in range(2, 200):
        r = pow(cand, (p - 1) // 16, p)
        if pow(r, 8, p) != 1:
            w = r
            break
    assert w is not None and pow(w, 16, p) == 1
    wi = pow(w, p - 2, p)
    E = [[pow(w, (brev4(j) * k) % 16, p) if forward else pow(wi, (j * brev4(k)) % 16, p) for k in range(16)]
         for j in range(16)]
    C = [[[E[j][k] * pow(2, 8 * s + 32, p) % p for s in range(4)] for k in range(16)] for j in range(16)]
    mont = (-pow(p, -1, 1 << 32)) % (1 << 32)
    rng = np.random.default_rng(p % 1000 + forward)
    for trial in range(20):
        x = [int(v) for v in rng.integers(0, 2**32, 16)]  # any 32-bit words
        if trial == 0:
            x = [0xFFFFFFFF] * 16  # the largest bytes
        for j in range(16):
            D = [sum(((C[j][k][s] >> (8 * l)) & 255) * ((x[k] >> (8 * s)) & 255) for k in range(16) for s in range(4))
                 for l in range(4)]
            assert all(d <= 64 * 255 * 255 < 1 << 22 for d in D)
            V = sum(d << (8 * l) for l, d in enumerate(D))
            assert V < 1 << 46 < p << 32
            assert V % p == (sum(E[j][k] * x[k] for k in range(16)) << 32) % p
            # REDC: (V + m p) / 2^32 with m = (V mod 2^32) (-p^-1) mod 2^32
            m = ((V & 0xFFFFFFFF) * mont) & 0xFFFFFFFF
            r = (V + m * p) >> 32
            assert (V + m * p) % (1 << 32) == 0 and r < 2 * p
            assert r % p == sum(E[j][k] * x[k] for k in range(16)) % p


def _eval_mod_q(coeffs, t):
    acc = 0
    for c in reversed(coeffs):
        acc = (acc * t + c) % Q
    return acc


def test_result_check_catches_errors_nonzero_mod_q_and_misses_multiples_of_q():
    """What the randomised check can and cannot see: it compares c(t) with
    a(t) b(t) modulo q, so an error polynomial e = c' - a*b is seen exactly
    when e(t) != 0 mod q.  A single changed limb adds +-2^(32 l) to one
    coefficient, never 0 mod q (q is an odd prime), so e is a non-zero
    polynomial mod q and has at most deg(e) roots; an error that is a
    multiple of q in every coefficient is invisible at every t."""
    rng = np.random.default_rng(61)
    a = [int(v) for v in rng.integers(-2**62, 2**62, 9)]
    b = [int(v) for v in rng.integers(-2**62, 2**62, 7)]
    c = [sum(a[i] * b[k - i] for i in range(len(a)) if 0 <= k - i < len(b)) for k in range(len(a) + len(b) - 1)]
    ts = [int(v) for v in rng.integers(2, Q - 1, 8)]
    for t in ts:
        assert _eval_mod_q(c, t) == _eval_mod_q(a, t) * _eval_mod_q(b, t) % Q
    # one changed limb (limb l of coefficient k): caught at every sampled t
    for k, l in [(0, 0), (5, 3), (14, 1)]:
        bad = list(c)
        bad[k] += 1 << (32 * l)
        assert (1 << (32 * l)) % Q != 0
        assert all(_eval_mod_q(bad, t) != _eval_mod_q(a, t) * _eval_mod_q(b, t) % Q for t in ts)
    # a sign flipped on a coefficient equal to a multiple of q (error -2 c_k,
    # 0 mod q) and an error of q y^3: never caught
    bad = list(c)
    bad[3] += 5 * Q
    for t in ts:
        assert _eval_mod_q(bad, t) == _eval_mod_q(c, t)
    cq = list(c)
    cq[4] = 7 * Q
    flipped = list(cq)
    flipped[4] = -cq[4]
    for t in ts:
        assert _eval_mod_q(flipped, t) == _eval_mod_q(cq, t)


# ---------------------------------------------------------------------------
# The big-prime form (csrc/ipm_bigp.cu): arithmetic modulo the generalized
# Fermat prime p = r^2 + 1, r = 2^63 + 2^53 (the first prime of the paper's
# table in §3.1).
# ---------------------------------------------------------------------------

GF_R = 2**63 + 2**53
GF_P = GF_R * GF_R + 1


def _gf_divmod_r(x):
    """x = q r + m: a shift by 53 and two 64-bit divisions by 1025."""
    t = x >> 53
    hi, lo = t >> 32, t & 0xFFFFFFFF
    qh, rh = hi // 1025, hi % 1025
    assert (rh << 32 | lo) < 2**64 and hi < 2**64
    q = (qh << 32) + (rh << 32 | lo) // 1025
    return q, x - q * GF_R


def _gf_mul(x, y):
    x1, x0 = _gf_divmod_r(x)
    y1, y0 = _gf_divmod_r(y)
    A0, A2, B = x0 * y0, x1 * y1, x0 * y1 + x1 * y0
    assert max(x1, y1) <= GF_R < 2**64 and max(x0, y0) < GF_R and B < 2**128
    Bq, B0 = _gf_divmod_r(B)
    T, U = A0 + B0 * GF_R, A2 + Bq
    assert T < 2 * GF_P < 2**128 and U < 2 * GF_P
    T, U = T % GF_P, U % GF_P  # one conditional subtraction each
    return (T - U) % GF_P


def test_generalized_fermat_prime_facts():
    assert GF_R == 1025 * 2**53
    assert pow(3, (GF_P - 1) // 2, GF_P) == GF_P - 1  # 3 is a non-residue: 3^((p-1)/2^k) has order 2^k
    assert (GF_P - 1) % 2**106 == 0 and ((GF_P - 1) >> 106) % 2 == 1
    assert pow(GF_R, 2, GF_P) == GF_P - 1  # r^2 = -1: r is a primitive 4th root
    for a in (2, 3, 5, 7, 11, 13):  # Fermat tests (the table lists p as prime)
        assert pow(a, GF_P - 1, GF_P) == 1


def test_divmod_by_r_and_the_folded_product():
    rng = np.random.default_rng(126)
    xs = [0, 1, GF_R - 1, GF_R, GF_R + 1, GF_P - 1, GF_P - 2, 2**127 - 1] + \
         [int.from_bytes(rng.bytes(16), "little") % GF_P for _ in range(300)]
    for x in xs:
        q, m = _gf_divmod_r(x)
        assert 0 <= m < GF_R and q * GF_R + m == x
    for x in xs[:40]:
        for y in xs[-40:]:
            if x < GF_P and y < GF_P:
                assert _gf_mul(x, y) == x * y % GF_P
    big = [2**128 - 1, 2 * GF_R * (GF_R + 1) - 1]
    for x in big:
        q, m = _gf_divmod_r(x)
        assert q * GF_R + m == x and m < GF_R and q < 2**66
