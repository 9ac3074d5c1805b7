"""The Kronecker-substitution family (ks=1; §1 and §4, the comparison
method KS_s): c is read off the integer product a(2^s) b(2^s), computed as
the transform product of the operands' 32-bit digit polynomials, and its
signed slots are unpacked without a carry chain across slots.  Whole
outputs against the oracle, bit for bit: random and unbalanced shapes,
single coefficients, zeros, every sign pattern, the largest magnitudes
(where slots are fullest), cancellation to zero, and equality with the
default transform path.  Errors: a coefficient above its bit bound is
reported; shapes beyond the transform's length limit are refused by the
planner."""
import numpy as np
import pytest

import oracle
import paper_1612_05778_gb300 as ipm
import workloads as W
from bigint_util import from_ints, to_ints

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_05778_gb300 import build
    build.build()


def ks_mul(a, b, ba, bb, **kw):
    na, nb = a[0].shape[0], b[0].shape[0]
    plan = ipm.Plan((na, nb, ba, bb), flags=ipm.IPM_SYNC, ks=1, **kw)
    assert plan.info["ks"] == 1 and plan.info["ks_w"] == plan.info["lc"] + 3
    da, dan = ipm.to_device(*a)
    db, dbn = ipm.to_device(*b)
    c, cn = plan.empty_output()
    c.fill_(-1)
    cn.fill_(7)
    plan.mul(da, dan, db, dbn, c, cn)
    torch.cuda.synchronize()
    plan.sync()
    out = ipm.to_host(c, cn)
    lc = plan.info["lc"]
    plan.close()
    return out, lc


def assert_oracle(a, b, ba, bb, **kw):
    got, lc = ks_mul(a, b, ba, bb, **kw)
    want = oracle.polymul(a, b, lc)
    bad = np.nonzero((got[0] != want[0]).any(axis=1) | (got[1] != want[1]))[0]
    assert bad.size == 0, "mismatch at %s" % bad[:10].tolist()
    return got


SHAPES = [(1, 1, 1, 1), (1, 9, 32, 7), (9, 1, 7, 32), (3, 2, 33, 64), (17, 5, 1000, 31), (64, 64, 64, 64),
          (100, 3, 4096, 300), (257, 129, 95, 97), (1024, 1024, 255, 255), (700, 1500, 1000, 64),
          (2, 2, 16384, 16384), (2048, 2048, 2048, 2048)]


@pytest.mark.parametrize("na,nb,ba,bb", SHAPES)
def test_random_shapes(na, nb, ba, bb):
    rng = np.random.default_rng(na * 131 + nb * 7 + ba)
    assert_oracle(W.random_poly(rng, na, ba), W.random_poly(rng, nb, bb), ba, bb)


@pytest.mark.parametrize("neg_a,neg_b", [(False, False), (True, False), (True, True)])
def test_largest_magnitudes(neg_a, neg_b):
    """Every coefficient +-(2^bits - 1): the largest |c_t|, nearest to the
    slot boundary."""
    n, bits = 300, 500
    a = W.constant_poly(n, bits, negative=neg_a)
    b = W.constant_poly(n + 17, bits, negative=neg_b)
    got = assert_oracle(a, b, bits, bits)
    assert all(s == int(neg_a != neg_b) for s in got[1])


def test_alternating_signs_zeros_and_cancellation():
    vals_a = [0, -1, (1 << 200) - 1, 0, -(1 << 199), 5, 0, 0]
    vals_b = [-(1 << 200) + 1, 0, 3, -3, 0, (1 << 200) - 1]
    a, b = from_ints(vals_a, 7), from_ints(vals_b, 7)
    got = assert_oracle(a, b, 224, 224)
    # (y - 1)(y + 1) with huge equal magnitudes: c_1 cancels to +0
    big = (1 << 1000) - 77
    a2, b2 = from_ints([-big, big], 32), from_ints([big, big], 32)
    got2, _ = ks_mul(a2, b2, 1024, 1024)
    assert to_ints(*got2) == [-big * big, 0, big * big] and got2[1][1] == 0
    assert got[0].shape[0] == len(vals_a) + len(vals_b) - 1


def test_zero_polynomials():
    z = W.random_poly(np.random.default_rng(1), 50, 100)
    z[0][:] = 0
    z[1][:] = 1  # -0 on input is accepted
    b = W.random_poly(np.random.default_rng(2), 40, 90)
    got = assert_oracle(z, b, 100, 90)
    assert not got[0].any() and not got[1].any()


def test_same_bytes_as_the_default_path():
    rng = np.random.default_rng(9)
    na, nb, ba, bb = 1000, 777, 333, 444
    a, b = W.random_poly(rng, na, ba), W.random_poly(rng, nb, bb)
    got, _ = ks_mul(a, b, ba, bb)
    plan = ipm.Plan((na, nb, ba, bb), flags=ipm.IPM_SYNC)
    c, cn = plan.mul(*ipm.to_device(*a), *ipm.to_device(*b))
    torch.cuda.synchronize()
    ref = ipm.to_host(c, cn)
    plan.close()
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_digit_product_overrides_keep_the_result():
    rng = np.random.default_rng(4)
    a, b = W.random_poly(rng, 500, 256), W.random_poly(rng, 600, 256)
    ref, _ = ks_mul(a, b, 256, 256)
    for kw in ({"K": 4}, {"K": 8, "s": 2}):
        got, _ = ks_mul(a, b, 256, 256, **kw)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), kw


def test_bound_violation_is_reported():
    a = W.constant_poly(10, 64)
    b = W.constant_poly(10, 64)
    plan = ipm.Plan((10, 10, 40, 64), ks=1)
    c, cn = plan.mul(*ipm.to_device(*a), *ipm.to_device(*b))
    with pytest.raises(ipm.IpmError) as e:
        plan.sync()
    assert e.value.status == 2  # IPM_ERR_BOUND
    plan.close()


def test_beyond_the_length_limit_is_refused():
    with pytest.raises(ipm.IpmError) as e:
        ipm.Plan((4096, 4096, 4096, 4096), ks=1)
    assert e.value.status == 6  # IPM_ERR_UNSUPPORTED
