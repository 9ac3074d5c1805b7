"""GPU parity of the Taylor shift by one (ipm_taylor_shift, g(x) = f(x+1))
against the oracle (oracle/taylor.py: g_k = sum_{i>=k} C(i, k) f_i with
Python integers), bit-exact on every limb and sign.

Small and mid sizes compare whole outputs; the large case (2^14
coefficients of 4096 bits, every level's product on the transform path)
is checked on sampled coefficients computed one by one, on the exact
identity g(t) = f(t + 1) modulo three 61-bit primes at random t, and the
all-(2^bits - 1) input against its closed form g_k = (2^bits - 1) C(n, k+1).
"""
import math

import numpy as np
import pytest

import oracle
import paper_1612_05778_gb300 as ipm
import workloads as W
from bigint_util import CHECK_PRIMES, from_ints, to_ints
from oracle.taylor import taylor_coeffs, taylor_shift1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_05778_gb300 import build
    build.build()


def gpu_shift(f, bits, flags=0):
    n = f[0].shape[0]
    ts = ipm.TaylorShift(n, bits, flags=ipm.IPM_SYNC | flags)
    df, dfn = ipm.to_device(*f)
    g, gn = ts.shift(df, dfn)
    torch.cuda.synchronize()
    ts.sync()
    out = ipm.to_host(g, gn)
    limbs = ts.limbs
    ts.close()
    return out, limbs


# n <= 64 runs every level through products; n > 64 runs levels 0..5 in
# shared memory first, unless the coefficients are too wide for it (9000 bits)
@pytest.mark.parametrize("n,bits", [(1, 5), (2, 1), (3, 64), (8, 255), (64, 100), (65, 100), (100, 300), (257, 31),
                                    (513, 1000), (1024, 255), (200, 9000)])
def test_taylor_matches_oracle(n, bits):
    rng = np.random.default_rng(n * 13 + bits)
    f = W.random_poly(rng, n, bits)
    (g, gn), L = gpu_shift(f, bits)
    assert L == (bits + n + 31) // 32
    want = taylor_shift1(to_ints(*f))
    assert to_ints(g, gn) == want
    # limbs above each magnitude are zero and zero is +0
    assert all(gn[k] == 0 for k in range(n) if want[k] == 0)


def test_taylor_monomial_binomials():
    n = 300
    f = from_ints([0] * (n - 1) + [1], 1)
    (g, gn), _ = gpu_shift(f, 1)
    assert to_ints(g, gn) == [math.comb(n - 1, k) for k in range(n)]


@pytest.mark.parametrize("negative", [False, True])
def test_taylor_extreme_closed_form(negative):
    """Every coefficient +-(2^bits - 1): g_k = +-(2^bits - 1) C(n, k + 1),
    the largest magnitudes the output bound allows."""
    n, bits = 1000, 200
    f = W.constant_poly(n, bits, negative=negative)
    (g, gn), _ = gpu_shift(f, bits)
    s = -1 if negative else 1
    alpha = (1 << bits) - 1
    assert to_ints(g, gn) == [s * alpha * math.comb(n, k + 1) for k in range(n)]


def test_taylor_negative_zero_and_sparse():
    vals = [0, -5, 0, 0, 1 << 90, 0, -(1 << 100) + 7]
    f = from_ints(vals, 4)
    f[1][0] = 1  # -0
    (g, gn), _ = gpu_shift(f, 101)
    want = taylor_shift1(vals)
    assert to_ints(g, gn) == want
    assert all(gn[k] == 0 for k in range(len(vals)) if want[k] == 0)


@pytest.mark.parametrize("n", [64, 300])
def test_taylor_bound_violation_reported(n):
    rng = np.random.default_rng(8)
    f = W.random_poly(rng, n, 40)
    f[0][10, 1] |= 1 << 12  # bit 44 set, above the 40-bit bound
    ts = ipm.TaylorShift(n, 40)
    df, dfn = ipm.to_device(*f)
    ts.shift(df, dfn)
    with pytest.raises(ipm.IpmError) as e:
        ts.sync()
    assert e.value.status == 2
    ts.close()


def test_taylor_with_tensor_stages_equal():
    rng = np.random.default_rng(9)
    f = W.random_poly(rng, 700, 500)
    a, _ = gpu_shift(f, 500)
    b, _ = gpu_shift(f, 500, ipm.IPM_TENSOR_STAGES)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_taylor_large():
    """2^14 coefficients of 4096 bits (seed 5): the workload bench.py times."""
    sh, f = W.taylor_dense(seed=5)
    n, bits = sh
    (g, gn), L = gpu_shift(f, bits)
    F = to_ints(*f)
    ks = [0, 1, n // 2, n - 2, n - 1] + np.random.default_rng(1).integers(0, n, 2).tolist()
    got = to_ints(g[ks], gn[ks])
    assert got == taylor_coeffs(F, ks)
    rng = np.random.default_rng(2)
    for q in CHECK_PRIMES:
        t = int(rng.integers(2, 2**60))
        assert oracle.eval_mod((g, gn), t, q) == oracle.eval_mod(f, (t + 1) % q, q)
