"""The randomised product check (ipm_validate and the IPM_VALIDATE plan
flag): c(t) = a(t) b(t) modulo 2^61 - 1 at a random point.  The exact
products of every family pass; outputs corrupted on the host side -- one
bit of one limb, one sign, two coefficients swapped, a zeroed row -- fail.
No fault is made on the GPU: the corruption is an ordinary write to the
output tensor before the check runs."""
import numpy as np
import pytest

import oracle
import paper_1612_05778_gb300 as ipm
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_05778_gb300 import build
    build.build()


def product(na, nb, ba, bb, seed, flags=0, **kw):
    rng = np.random.default_rng(seed)
    a = W.random_poly(rng, na, ba)
    b = W.random_poly(rng, nb, bb)
    plan = ipm.Plan((na, nb, ba, bb), flags=flags, **kw)
    da, dan = ipm.to_device(*a)
    db, dbn = ipm.to_device(*b)
    c, cn = plan.mul(da, dan, db, dbn)
    plan.sync()
    plan.close()
    return (a, b), (da, dan, db, dbn), (c, cn)


SHAPES = [(1, 1, 1, 1, {}), (17, 5, 1000, 31, {}), (300, 250, 255, 255, {}), (3000, 2100, 700, 900, {}),
          (2000, 2000, 16, 16, {"kron": 4}), (40, 60, 200, 100, {"school": 1}), (300, 250, 255, 255, {"y1b": 4})]


@pytest.mark.parametrize("na,nb,ba,bb,kw", SHAPES)
def test_exact_products_pass(na, nb, ba, bb, kw):
    (a, b), d, (c, cn) = product(na, nb, ba, bb, na + nb, **kw)
    for seed in (1, 2, 3):
        assert ipm.validate(na, nb, ba, bb, *d, c, cn, seed=seed)


@pytest.mark.parametrize("what", ["bit", "sign", "swap", "zero_row", "top_limb"])
def test_corrupted_outputs_fail(what):
    na, nb, ba, bb = 700, 500, 300, 200
    (a, b), d, (c, cn) = product(na, nb, ba, bb, 5)
    assert ipm.validate(na, nb, ba, bb, *d, c, cn)
    c2, cn2 = c.clone(), cn.clone()
    if what == "bit":
        c2[333, 4] ^= 1 << 17
    elif what == "sign":
        k = int(torch.nonzero(c2.abs().sum(dim=1))[10])
        cn2[k] ^= 1
    elif what == "swap":
        c2[[100, 101]] = c2[[101, 100]]
        cn2[[100, 101]] = cn2[[101, 100]]
        assert not torch.equal(c2, c)
    elif what == "zero_row":
        c2[600] = 0
    else:
        c2[0, -1] ^= 1 << 31
    for seed in (1, 2):
        assert not ipm.validate(na, nb, ba, bb, *d, c2, cn2, seed=seed)


def test_plan_flag_checks_every_product():
    """IPM_VALIDATE on single products, device and host buffers, and on the
    full-size benchmarked workload (two degree-32767 polynomials with
    4096-bit coefficients): no false alarms."""
    for shape in [(300, 250, 255, 255), (1, 9, 64, 64), (4097, 1000, 300, 33)]:
        for _ in range(2):
            product(*shape, seed=sum(shape), flags=ipm.IPM_VALIDATE)
    rng = np.random.default_rng(3)
    a = W.random_poly(rng, 500, 100)
    b = W.random_poly(rng, 400, 90)
    plan = ipm.Plan((500, 400, 100, 90), flags=ipm.IPM_VALIDATE)
    c, cn = plan.mul_host(a[0], a[1], b[0], b[1])
    want = oracle.polymul(a, b, plan.info["lc"])
    assert np.array_equal(c, want[0]) and np.array_equal(cn, want[1])
    plan.close()
    sh, a, b = W.large_dense(seed=1)
    plan = ipm.Plan((sh.na, sh.nb, sh.bits_a, sh.bits_b), flags=ipm.IPM_VALIDATE)
    da, dan = ipm.to_device(*a)
    db, dbn = ipm.to_device(*b)
    plan.mul(da, dan, db, dbn)
    plan.sync()
    plan.close()


def _batch(seed, count):
    shapes = W.batch_shapes(seed=seed, count=count, dmin=16, dmax=900, bmin=32, bmax=700)
    ops = W.batch_operands(shapes, seed=seed)
    dev = [ipm.to_device(*a) + ipm.to_device(*b) for a, b in ops]
    return shapes, ops, dev


@pytest.mark.parametrize("flags", [ipm.IPM_VALIDATE, ipm.IPM_VALIDATE | ipm.IPM_GRAPH])
def test_batched_check_passes_exact_products(flags):
    """Every product of a batched call checked in two launches, including
    products that run alone (split middle transform, packed, schoolbook)."""
    shapes, ops, dev = _batch(21, 14)
    tuples = [(s.na, s.nb, s.bits_a, s.bits_b) for s in shapes]
    plan = ipm.Plan(tuples, flags=flags)
    for _ in range(2):
        outs = plan.mul_batched(dev)
        plan.sync()
    for (a, b), (c, cn), info in zip(ops, outs, plan.infos):
        want = oracle.polymul(a, b, info["lc"])
        got = ipm.to_host(c, cn)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    plan.close()


def test_batched_check_catches_a_shared_output():
    """Two products of one batched call handed the same output buffer (a
    caller's mistake, made on the host): the buffer cannot hold both
    products, and the check reports IPM_ERR_MISMATCH."""
    rng = np.random.default_rng(31)
    shape = (200, 150, 100, 90)
    ops = [(W.random_poly(rng, 200, 100), W.random_poly(rng, 150, 90)) for _ in range(3)]
    dev = [ipm.to_device(*a) + ipm.to_device(*b) for a, b in ops]
    plan = ipm.Plan([shape] * 3, flags=ipm.IPM_VALIDATE)
    outs = [plan.empty_output(i) for i in range(3)]
    outs[1] = outs[0]
    plan.mul_batched(dev, outs)
    with pytest.raises(ipm.IpmError) as e:
        plan.sync()
    assert e.value.status == 7
    # separate buffers again: no alarm
    outs = [plan.empty_output(i) for i in range(3)]
    plan.mul_batched(dev, outs)
    plan.sync()
    plan.close()
