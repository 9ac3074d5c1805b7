"""GPU parity of Kronecker balancing (the paper's §3 footnote): products of
packed operands decoded back into exact coefficients, bit-exact against the
CPU oracle on every limb and sign.

Cases: every packing factor; coefficient counts that are not multiples of
the factor, unbalanced pairs, fewer coefficients than the factor; extreme
magnitudes (every coefficient +-(2^bits - 1), which drives every slot to
its bound); slot widths up to the 128-bit limit; zero polynomials;
inner plans with K halved and doubled; a batched call mixing packed and
unpacked products; a bound violation reported through the packing kernel.
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


def check(a, b, ba, bb, **kw):
    got, info = gpu_mul(a, b, ba, bb, **kw)
    assert info["kron"] == kw.get("kron", 1)
    assert_same(got, oracle.polymul(a, b, info["lc"]))
    return info


@pytest.mark.parametrize("s", [2, 4, 8, 16])
@pytest.mark.parametrize("na,nb,ba,bb", [(1000, 1000, 32, 32), (777, 1234, 20, 40), (3001, 95, 48, 8),
                                         (5, 3, 32, 32), (1, 40, 16, 16)])
def test_packed_matches_oracle(s, na, nb, ba, bb):
    rng = np.random.default_rng(na * 13 + nb + s)
    a = W.random_poly(rng, na, ba)
    b = W.random_poly(rng, nb, bb)
    info = check(a, b, ba, bb, kron=s)
    assert info["kron_na"] == -(-na // s) and info["kron_nb"] == -(-nb // s)


@pytest.mark.parametrize("s", [2, 8, 16])
@pytest.mark.parametrize("signs", ["positive", "negative", "alternating"])
def test_extreme_magnitudes(s, signs):
    """Every coefficient of magnitude 2^bits - 1: the slot sums reach their
    bound min(na, nb) (2^bits_a - 1)(2^bits_b - 1)."""
    na, nb, ba, bb = 1024, 1024, 33, 31
    va = (1 << ba) - 1
    vb = (1 << bb) - 1
    if signs == "positive":
        A, B = [va] * na, [vb] * nb
    elif signs == "negative":
        A, B = [-va] * na, [vb] * nb
    else:
        A = [va if i % 2 else -va for i in range(na)]
        B = [-vb if i % 3 else vb for i in range(nb)]
    check(from_ints(A, 2), from_ints(B, 1), ba, bb, kron=s)


def test_slot_width_limit():
    """bits_a + bits_b + ceil(log2 min(na, nb)) + 1 = 128, the widest slot."""
    na = nb = 2048  # log2 = 11
    ba, bb = 58, 58  # w = 58 + 58 + 11 + 1 = 128
    rng = np.random.default_rng(8)
    a = W.random_poly(rng, na, ba)
    b = W.random_poly(rng, nb, bb)
    info = check(a, b, ba, bb, kron=4)
    assert info["kron_w"] == 128
    with pytest.raises(ipm.IpmError):
        ipm.Plan((na, nb, ba + 1, bb), kron=4)


@pytest.mark.parametrize("K", [8, 16, 64])
def test_inner_plan_invariance(K):
    rng = np.random.default_rng(21)
    a = W.random_poly(rng, 900, 30)
    b = W.random_poly(rng, 700, 30)
    check(a, b, 30, 30, kron=4, K=K)


def test_zero_and_sparse():
    a = (np.zeros((40, 1), np.uint32), np.zeros(40, np.uint8))
    b = W.random_poly(np.random.default_rng(2), 33, 32)
    (c, cn), _ = gpu_mul(a, b, 32, 32, kron=8)
    assert not c.any() and not cn.any()
    vals = [0] * 50
    vals[17] = -5
    vals[49] = 3
    check(from_ints(vals, 1), from_ints([0, 0, 0, 7, -1, 0, 2], 1), 4, 4, kron=4)


def test_batched_mixes_packed_and_plain_products():
    """Per-shape plans come from the tuning table (IPM_COSTMODEL): three
    packed products and one plain one in a single batched call."""
    shapes = [(300, 200, 32, 32), (1000, 1000, 24, 24), (64, 5000, 16, 20), (400, 400, 300, 300)]
    rng = np.random.default_rng(31)
    ops = [(W.random_poly(rng, na, ba), W.random_poly(rng, nb, bb)) for na, nb, ba, bb in shapes]
    ipm.set_tuned([(sh, {"kron": 4}) for sh in shapes[:3]])
    try:
        plan = ipm.Plan(shapes, flags=ipm.IPM_SYNC | ipm.IPM_COSTMODEL)
    finally:
        ipm.set_tuned([])
    assert [i["kron"] for i in plan.infos] == [4, 4, 4, 1]
    dev = [ipm.to_device(*a) + ipm.to_device(*b) for a, b in ops]
    outs = plan.mul_batched(dev)
    torch.cuda.synchronize()
    for (a, b), (c, cn), info in zip(ops, outs, plan.infos):
        assert_same(ipm.to_host(c, cn), oracle.polymul(a, b, info["lc"]))


def test_bound_violation_through_packing():
    rng = np.random.default_rng(3)
    a = W.random_poly(rng, 64, 20)
    b = W.random_poly(rng, 64, 20)
    a[0][9, 0] |= 1 << 25  # above the 20-bit bound
    plan = ipm.Plan((64, 64, 20, 20), kron=4)
    da, dan = ipm.to_device(*a)
    db, dbn = ipm.to_device(*b)
    plan.mul(da, dan, db, dbn)
    with pytest.raises(ipm.IpmError) as e:
        plan.sync()
    assert e.value.status == 2
