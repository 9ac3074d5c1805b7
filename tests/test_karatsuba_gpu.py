"""The Karatsuba family (kara=L): L levels of Karatsuba's three-product
recursion over y with the schoolbook kernel at the 3^L leaves, every
level's combination on the GPU.  Whole outputs against the oracle, bit for
bit: every level count, balanced and unbalanced degrees (padding), odd
lengths, single coefficients, the largest magnitudes (the leaf operand
sums a0 + a1 reach bits + L), all-negative and alternating signs, zero
polynomials and cancellation; equality with the default path; a bound
violation is reported."""
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


def kara_mul(a, b, ba, bb, levels):
    na, nb = a[0].shape[0], b[0].shape[0]
    plan = ipm.Plan((na, nb, ba, bb), flags=ipm.IPM_SYNC, kara=levels)
    assert plan.info["kara"] == levels
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


def assert_oracle(a, b, ba, bb, levels):
    got, lc = kara_mul(a, b, ba, bb, levels)
    want = oracle.polymul(a, b, lc)
    bad = np.nonzero((got[0] != want[0]).any(axis=1) | (got[1] != want[1]))[0]
    assert bad.size == 0, "mismatch at %s" % bad[:10].tolist()
    return got


SHAPES = [(1, 1, 1, 1), (2, 2, 64, 64), (3, 1, 33, 7), (17, 5, 1000, 31), (64, 64, 64, 64),
          (100, 3, 4096, 300), (257, 129, 95, 97), (1000, 1000, 255, 255), (700, 1500, 1000, 64)]


@pytest.mark.parametrize("levels", [1, 2, 3, 4])
@pytest.mark.parametrize("na,nb,ba,bb", SHAPES)
def test_random_shapes(na, nb, ba, bb, levels):
    rng = np.random.default_rng(na * 17 + nb * 3 + ba + levels)
    assert_oracle(W.random_poly(rng, na, ba), W.random_poly(rng, nb, bb), ba, bb, levels)


@pytest.mark.parametrize("levels", [1, 3])
@pytest.mark.parametrize("neg_a,neg_b", [(False, False), (True, False), (True, True)])
def test_largest_magnitudes(levels, neg_a, neg_b):
    """Every coefficient +-(2^bits - 1): the leaf sums and the node products
    are at their bounds."""
    a = W.constant_poly(200, 500, negative=neg_a)
    b = W.constant_poly(333, 500, negative=neg_b)
    got = assert_oracle(a, b, 500, 500, levels)
    assert all(s == int(neg_a != neg_b) for s in got[1])


@pytest.mark.parametrize("levels", [2, 4])
def test_signs_zeros_and_cancellation(levels):
    vals_a = [0, -1, (1 << 200) - 1, 0, -(1 << 199), 5, 0, 0, 7, -7, 1 << 100]
    vals_b = [-(1 << 200) + 1, 0, 3, -3, 0, (1 << 200) - 1]
    assert_oracle(from_ints(vals_a, 7), from_ints(vals_b, 7), 224, 224, levels)
    big = (1 << 1000) - 77
    got, _ = kara_mul(from_ints([-big, big], 32), from_ints([big, big], 32), 1024, 1024, levels)
    assert to_ints(*got) == [-big * big, 0, big * big] and got[1][1] == 0
    z = W.random_poly(np.random.default_rng(1), 50, 100)
    z[0][:] = 0
    z[1][:] = 1  # -0 on input is accepted
    got = assert_oracle(z, W.random_poly(np.random.default_rng(2), 41, 90), 100, 90, levels)
    assert not got[0].any() and not got[1].any()


def test_same_bytes_as_the_default_path():
    rng = np.random.default_rng(9)
    na, nb, ba, bb = 1024, 800, 512, 300
    a, b = W.random_poly(rng, na, ba), W.random_poly(rng, nb, bb)
    got, _ = kara_mul(a, b, ba, bb, 3)
    plan = ipm.Plan((na, nb, ba, bb), flags=ipm.IPM_SYNC)
    c, cn = plan.mul(*ipm.to_device(*a), *ipm.to_device(*b))
    torch.cuda.synchronize()
    ref = ipm.to_host(c, cn)
    plan.close()
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_bound_violation_is_reported():
    a = W.constant_poly(40, 64)
    plan = ipm.Plan((40, 40, 40, 64), kara=2)
    plan.mul(*ipm.to_device(*a), *ipm.to_device(*a))
    with pytest.raises(ipm.IpmError) as e:
        plan.sync()
    assert e.value.status == 2  # IPM_ERR_BOUND
    plan.close()


def test_in_a_batched_call():
    """Karatsuba products run one by one after the grouped launches of a
    batched call; the results are the same exact products."""
    shapes = W.batch_shapes(seed=11, count=4, dmin=20, dmax=300, bmin=32, bmax=500)
    ops = W.batch_operands(shapes, seed=11)
    plan = ipm.Plan([(s.na, s.nb, s.bits_a, s.bits_b) for s in shapes], flags=ipm.IPM_SYNC, kara=2)
    dev = [ipm.to_device(*a) + ipm.to_device(*b) for a, b in ops]
    outs = plan.mul_batched(dev)
    torch.cuda.synchronize()
    for s, (a, b), (c, cn) in zip(shapes, ops, outs):
        want = oracle.polymul(a, b, s.lc)
        got = ipm.to_host(c, cn)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    plan.close()
