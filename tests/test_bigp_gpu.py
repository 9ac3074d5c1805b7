"""The big-prime form (bigp=1; §3.1 and §4): the cyclic and negacyclic
convolutions of §2.1 modulo one generalized Fermat prime p = (2^63 +
2^53)^2 + 1, no Chinese remaindering.  Whole outputs against the oracle,
bit for bit: random and unbalanced shapes, single coefficients, zeros,
every sign pattern, the largest magnitudes, cancellation, overridden K,
equality with the word-prime path; a bound violation is reported and
shapes whose bound exceeds p are refused."""
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


def bigp_mul(a, b, ba, bb, **kw):
    na, nb = a[0].shape[0], b[0].shape[0]
    plan = ipm.Plan((na, nb, ba, bb), flags=ipm.IPM_SYNC, bigp=1, **kw)
    assert plan.info["bigp"] == 1 and plan.info["r"] == 1
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
    got, lc = bigp_mul(a, b, ba, bb, **kw)
    want = oracle.polymul(a, b, lc)
    bad = np.nonzero((got[0] != want[0]).any(axis=1) | (got[1] != want[1]))[0]
    assert bad.size == 0, "mismatch at %s" % bad[:10].tolist()
    return got


SHAPES = [(1, 1, 1, 1), (1, 9, 32, 7), (9, 1, 7, 32), (3, 2, 33, 64), (17, 5, 1000, 31), (64, 64, 64, 64),
          (100, 3, 4096, 300), (257, 129, 95, 97), (1024, 1024, 255, 255), (700, 1500, 1000, 64),
          (2, 2, 16384, 16384), (2048, 2048, 2048, 2048)]


@pytest.mark.parametrize("na,nb,ba,bb", SHAPES)
def test_random_shapes(na, nb, ba, bb):
    rng = np.random.default_rng(na * 29 + nb * 5 + ba)
    assert_oracle(W.random_poly(rng, na, ba), W.random_poly(rng, nb, bb), ba, bb)


@pytest.mark.parametrize("neg_a,neg_b", [(False, False), (True, False), (True, True)])
def test_largest_magnitudes(neg_a, neg_b):
    a = W.constant_poly(300, 500, negative=neg_a)
    b = W.constant_poly(317, 500, negative=neg_b)
    got = assert_oracle(a, b, 500, 500)
    assert all(s == int(neg_a != neg_b) for s in got[1])


def test_signs_zeros_and_cancellation():
    vals_a = [0, -1, (1 << 200) - 1, 0, -(1 << 199), 5, 0, 0]
    vals_b = [-(1 << 200) + 1, 0, 3, -3, 0, (1 << 200) - 1]
    assert_oracle(from_ints(vals_a, 7), from_ints(vals_b, 7), 224, 224)
    big = (1 << 1000) - 77
    got, _ = bigp_mul(from_ints([-big, big], 32), from_ints([big, big], 32), 1024, 1024)
    assert to_ints(*got) == [-big * big, 0, big * big] and got[1][1] == 0
    z = W.random_poly(np.random.default_rng(1), 50, 100)
    z[0][:] = 0
    z[1][:] = 1  # -0 on input is accepted
    got = assert_oracle(z, W.random_poly(np.random.default_rng(2), 40, 90), 100, 90)
    assert not got[0].any() and not got[1].any()


@pytest.mark.parametrize("K", [16, 64, 256])
def test_overridden_K(K):
    rng = np.random.default_rng(K)
    assert_oracle(W.random_poly(rng, 333, 700), W.random_poly(rng, 222, 700), 700, 700, K=K)


def test_same_bytes_as_the_word_prime_path():
    rng = np.random.default_rng(9)
    na, nb, ba, bb = 1000, 777, 333, 444
    a, b = W.random_poly(rng, na, ba), W.random_poly(rng, nb, bb)
    got, _ = bigp_mul(a, b, ba, bb)
    plan = ipm.Plan((na, nb, ba, bb), flags=ipm.IPM_SYNC)
    c, cn = plan.mul(*ipm.to_device(*a), *ipm.to_device(*b))
    torch.cuda.synchronize()
    ref = ipm.to_host(c, cn)
    plan.close()
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_bound_violation_is_reported():
    a = W.constant_poly(10, 64)
    plan = ipm.Plan((10, 10, 40, 64), bigp=1)
    plan.mul(*ipm.to_device(*a), *ipm.to_device(*a))
    with pytest.raises(ipm.IpmError) as e:
        plan.sync()
    assert e.value.status == 2  # IPM_ERR_BOUND
    plan.close()
