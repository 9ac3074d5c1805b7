"""GPU parity of the schoolbook family (direct limb products, one block per
output coefficient), bit-exact against the CPU oracle on every limb and
sign: random, ragged and unbalanced shapes, bit bounds that are not
multiples of 32, extreme magnitudes of both signs, zero and single-term
operands, the family's column limit, a batched call mixing the schoolbook
and transform families, and a bound violation.
"""
import numpy as np
import pytest

import oracle
import paper_1612_05778_gb300 as ipm
import workloads as W
from bigint_util import from_ints

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_05778_gb300 import build
    build.build()


def gpu_mul(a, b, bits_a, bits_b, **kw):
    na, nb = a[0].shape[0], b[0].shape[0]
    plan = ipm.Plan((na, nb, bits_a, bits_b), flags=ipm.IPM_SYNC, **kw)
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


def check(a, b, ba, bb):
    got, info = gpu_mul(a, b, ba, bb, school=1)
    assert info["school"] == 1
    assert_same(got, oracle.polymul(a, b, info["lc"]))


@pytest.mark.parametrize("na,nb,ba,bb", [(64, 64, 32, 32), (300, 257, 255, 255), (1, 1, 1, 1), (1000, 3, 17, 900),
                                         (5, 777, 4096, 31), (129, 130, 96, 97), (2, 2048, 64, 64)])
def test_schoolbook_matches_oracle(na, nb, ba, bb):
    rng = np.random.default_rng(na * 7 + nb * 3 + ba + bb)
    check(W.random_poly(rng, na, ba), W.random_poly(rng, nb, bb), ba, bb)


@pytest.mark.parametrize("signs", ["positive", "negative", "mixed"])
def test_schoolbook_extremes(signs):
    na, nb, ba, bb = 200, 150, 200, 130
    va, vb = (1 << ba) - 1, (1 << bb) - 1
    if signs == "positive":
        A, B = [va] * na, [vb] * nb
    elif signs == "negative":
        A, B = [-va] * na, [vb] * nb
    else:
        A = [va if i % 2 else -va for i in range(na)]
        B = [-vb if i % 5 else vb for i in range(nb)]
    check(from_ints(A, 7), from_ints(B, 5), ba, bb)


def test_schoolbook_zero_and_single_terms():
    a = (np.zeros((40, 2), np.uint32), np.zeros(40, np.uint8))
    b = W.random_poly(np.random.default_rng(2), 33, 60)
    (c, cn), _ = gpu_mul(a, b, 60, 60, school=1)
    assert not c.any() and not cn.any()
    vals = [0] * 50
    vals[49] = -3
    check(from_ints(vals, 1), from_ints([0, 0, 0, 7], 1), 3, 3)


def test_schoolbook_limits():
    ipm.Plan((16, 16, 4096, 4096), school=1).close()       # La + Lb = 256
    with pytest.raises(ipm.IpmError):
        ipm.Plan((16, 16, 4096, 4097), school=1)          # 257 columns
    with pytest.raises(ipm.IpmError):
        ipm.Plan((1 << 14, 1 << 14, 32, 32), school=1)    # 2^28 limb products
    with pytest.raises(ipm.IpmError):
        ipm.Plan((64, 64, 32, 32), school=1, K=4)         # no transform overrides


def test_batched_mixes_families():
    shapes = [(100, 90, 64, 64), (2000, 1500, 300, 200), (7, 500, 33, 33), (600, 600, 24, 24)]
    rng = np.random.default_rng(41)
    ops = [(W.random_poly(rng, na, ba), W.random_poly(rng, nb, bb)) for na, nb, ba, bb in shapes]
    ipm.set_tuned([(shapes[0], {"school": 1}), (shapes[2], {"school": 1}), (shapes[3], {"kron": 8})])
    try:
        plan = ipm.Plan(shapes, flags=ipm.IPM_SYNC | ipm.IPM_COSTMODEL)
    finally:
        ipm.set_tuned([])
    assert [i["school"] for i in plan.infos] == [1, 0, 1, 0] and plan.infos[3]["kron"] == 8
    dev = [ipm.to_device(*a) + ipm.to_device(*b) for a, b in ops]
    outs = plan.mul_batched(dev)
    torch.cuda.synchronize()
    for (a, b), (c, cn), info in zip(ops, outs, plan.infos):
        assert_same(ipm.to_host(c, cn), oracle.polymul(a, b, info["lc"]))


def test_schoolbook_bound_violation():
    rng = np.random.default_rng(5)
    a = W.random_poly(rng, 30, 40)
    b = W.random_poly(rng, 30, 40)
    b[0][29, 1] |= 1 << 12  # bit 44, above the 40-bit bound
    plan = ipm.Plan((30, 30, 40, 40), school=1)
    da, dan = ipm.to_device(*a)
    db, dbn = ipm.to_device(*b)
    plan.mul(da, dan, db, dbn)
    with pytest.raises(ipm.IpmError) as e:
        plan.sync()
    assert e.value.status == 2
