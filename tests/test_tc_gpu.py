"""GPU parity of the tensor-core transform stages (plan flag
IPM_TENSOR_STAGES): every radix-16 stage of the forward, middle, outer and
inverse passes runs as byte-slice products on the INT8 tensor cores with
32-bit accumulation and an exact Montgomery reduction.  The output must be
the exact product: equal to the oracle on every limb and sign, and byte for
byte equal to the integer-stage path.

The plan overrides below are chosen so that each place a radix-16 stage
can occur is reached: the x DFTs (K = 16, 256, 2048), y step A with and
without a zero upper half (Y2 = 16, 256), the middle transform's forward
stages and its last inverse stage writing to the workspace (Y1 = 256,
1024, 2048), the outer pass of a split middle transform (Y1b = 16), and
the inverse pass's first y stage reading through the row twiddle.
"""
import numpy as np
import pytest

import oracle
import paper_1612_05778_gb300 as ipm
import workloads as W
from bigint_util import CHECK_PRIMES, eval_at, full_output_digest, stored_full_digest, to_ints

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_05778_gb300 import build
    build.build()


def gpu_mul(a, b, bits_a, bits_b, flags=0, **kw):
    na, nb = a[0].shape[0], b[0].shape[0]
    plan = ipm.Plan((na, nb, bits_a, bits_b), flags=ipm.IPM_SYNC | flags, **kw)
    da, dan = ipm.to_device(*a)
    db, dbn = ipm.to_device(*b)
    c, cn = plan.mul(da, dan, db, dbn)
    torch.cuda.synchronize()
    plan.sync()
    out = ipm.to_host(c, cn)
    info = plan.info
    plan.close()
    return out, info


def assert_same(got, want):
    gl, gn = got
    wl, wn = want
    assert gl.shape == wl.shape
    bad = np.nonzero((gl != wl).any(axis=1) | (gn != wn))[0]
    assert bad.size == 0, "mismatch at coefficients %s" % bad[:10].tolist()


def stage_bits(logL):
    """Radix exponents of the stages a length-2^logL transform uses."""
    nst = (logL + 3) // 4
    if nst == 0:
        return []
    base, extra = logL // nst, logL % nst
    return [base + (1 if i < extra else 0) for i in range(nst)]


CASES = [
    # (na, nb, bits_a, bits_b, overrides)
    (300, 250, 255, 255, dict(K=16, y2=16)),      # x: one radix-16 stage; y step A: zero upper half
    (300, 250, 255, 255, dict(K=16, y2=256)),     # y step A: two radix-16 stages
    (300, 250, 255, 255, dict(K=256)),            # x: two radix-16 stages
    (300, 250, 255, 255, dict(y2=4)),             # middle Y1 = 256: 16 x 16
    (300, 250, 255, 255, dict(y2=1)),             # middle Y1 = 1024: 16 x 8 x 8
    (2000, 2000, 64, 64, dict(y2=2)),             # middle Y1 = 2048: 16 x 16 x 8
    (300, 250, 255, 255, dict(y1b=16)),           # outer pass: Y1b = 16
    (40, 33, 4000, 3000, dict(K=2048, M=2)),      # x: 16 x 16 x 8
    (1500, 4000, 1024, 64, dict()),               # planner's plan, several tiles, ragged tail
    (129, 257, 95, 97, dict()),
    (1, 1, 1, 1, dict()),
    (5, 100, 31, 4096, dict()),
    (20000, 20000, 16, 16, dict(kron=8)),         # Kronecker-packed operands, middle Y1 = 256
]


@pytest.mark.parametrize("na,nb,ba,bb,kw", CASES)
def test_tensor_stages_match_oracle(na, nb, ba, bb, kw):
    rng = np.random.default_rng(na * 31 + nb + ba)
    a = W.random_poly(rng, na, ba)
    b = W.random_poly(rng, nb, bb)
    got, info = gpu_mul(a, b, ba, bb, ipm.IPM_TENSOR_STAGES, **kw)
    assert_same(got, oracle.polymul(a, b, info["lc"]))


def test_tensor_stages_digit_extreme():
    """Balanced digits all -2^(M-1): residues at the top of their range."""
    na = nb = 512
    bits = 1000
    info = ipm.choose(na, nb, bits, bits, K=32, y2=16)
    M = info["M"]
    half = 1 << (M - 1)
    mag = sum(half << (M * j) for j in range(bits // M))
    L = W.limbs_for_bits(bits)
    from bigint_util import from_ints
    a = from_ints([-mag] * na, L)
    b = from_ints([mag] * nb, L)
    got, info = gpu_mul(a, b, bits, bits, ipm.IPM_TENSOR_STAGES, K=32, y2=16)
    assert_same(got, oracle.polymul(a, b, info["lc"]))


def test_tensor_stages_bytes_equal_integer_path():
    rng = np.random.default_rng(77)
    a = W.random_poly(rng, 3000, 700)
    b = W.random_poly(rng, 2100, 900)
    got_tc, _ = gpu_mul(a, b, 700, 900, ipm.IPM_TENSOR_STAGES)
    got_int, _ = gpu_mul(a, b, 700, 900, 0)
    assert np.array_equal(got_tc[0], got_int[0]) and np.array_equal(got_tc[1], got_int[1])


def _identities(a, b, c):
    A, B, C = to_ints(*a), to_ints(*b), to_ints(*c)
    for t in (1, -1):
        assert eval_at(C, t) == eval_at(A, t) * eval_at(B, t)
    rng = np.random.default_rng(321)
    for q in CHECK_PRIMES:
        t = int(rng.integers(2, 2**60))
        assert oracle.eval_mod(c, t, q) == oracle.eval_mod(a, t, q) * oracle.eval_mod(b, t, q) % q


@pytest.mark.parametrize("which", ["large_dense", "huge_dense", "huge_mixed"])
def test_tensor_stages_full_size(which):
    """The benchmarked sizes: two degree-32767 polynomials of 4096-bit
    coefficients, and two degree-262143 polynomials of 1024-bit (or mixed
    64/2048-bit) coefficients -- sampled coefficients against the oracle,
    the exact identities C(+-1) = A(+-1)B(+-1), evaluation modulo three
    61-bit primes, and the whole output equal to the integer path's."""
    sh, a, b = getattr(W, which)(seed=1 if which == "large_dense" else 2)
    got, info = gpu_mul(a, b, sh.bits_a, sh.bits_b, ipm.IPM_TENSOR_STAGES)
    nc = sh.nc
    ks = [0, 1, 2, nc // 2, nc - 2, nc - 1] + np.random.default_rng(nc).integers(0, nc, 3).tolist()
    assert_same((got[0][ks], got[1][ks]), oracle.coeffs(ks, a, b, sh.lc))
    _identities(a, b, got)
    ref, _ = gpu_mul(a, b, sh.bits_a, sh.bits_b, 0)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    # every limb and sign against the oracle's whole product
    want = stored_full_digest(which)
    assert want is not None and full_output_digest(*got) == want
