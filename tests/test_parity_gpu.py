"""GPU parity: the CUDA path against the CPU oracle, bit-exact on every limb
and sign (integer work: exact equality is the only tolerance).

Small and mid sizes compare whole outputs with the oracle.  The full-size
workloads (two degree-32767 polynomials with 4096-bit coefficients; two of
degree 262143 with 1024-bit or mixed 64/2048-bit coefficients) are compared
on every limb and sign through the SHA-256 digest of the oracle's whole
product (Kronecker substitution with the oracle's own Karatsuba,
tests/golden/make_full_digests.py), with both the analytic planner's plan
and the plan bench.py times (the learned dispatch), and also on sampled
coefficients computed one by one by the oracle, on the exact identities
C(1) = A(1)B(1) and C(-1) = A(-1)B(-1), and on evaluation modulo three
independent 61-bit primes; the all-(2^4096-1) variant is checked in full
against the closed form c_k = terms(k) (2^4096-1)^2.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import paper_1612_05778_gb300 as ipm
import workloads as W
from bigint_util import (CHECK_PRIMES, eval_at, from_ints, full_output_digest, stored_full_digest, terms,
                         to_ints)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


def check_vs_oracle(a, b, ba, bb, **kw):
    got, info = gpu_mul(a, b, ba, bb, **kw)
    want = oracle.polymul(a, b, info["lc"])
    assert_same(got, want)
    return got, info


# ---- whole outputs against the oracle -------------------------------------

SMALL = [(1, 1, 1, 1), (1, 5, 32, 7), (5, 1, 7, 32), (3, 2, 33, 64), (7, 7, 100, 100),
         (17, 5, 1000, 31), (64, 64, 64, 64), (100, 3, 4096, 300), (5, 100, 31, 4096),
         (33, 33, 32, 32), (2, 2, 16384, 16384), (129, 257, 95, 97)]


@pytest.mark.parametrize("na,nb,ba,bb", SMALL)
def test_small_shapes(na, nb, ba, bb):
    rng = np.random.default_rng(na * 7919 + nb * 31 + ba + bb)
    a = W.random_poly(rng, na, ba)
    b = W.random_poly(rng, nb, bb)
    check_vs_oracle(a, b, ba, bb)


@pytest.mark.parametrize("na,nb,ba,bb", [(3000, 2100, 64, 200), (2049, 2049, 255, 255),
                                         (4097, 1000, 300, 33), (1500, 4000, 1024, 64)])
def test_multi_tile_ragged(na, nb, ba, bb):
    """Several tiles in every pass and a ragged tail of rows beyond n."""
    rng = np.random.default_rng(na + nb)
    a = W.random_poly(rng, na, ba)
    b = W.random_poly(rng, nb, bb)
    check_vs_oracle(a, b, ba, bb)


def test_small_dense_workload_full():
    """Two degree-1023 polynomials, |coeff| < 2^255, seed 0: every limb."""
    sh, a, b = W.small_dense(seed=0)
    got, info = check_vs_oracle(a, b, sh.bits_a, sh.bits_b)
    with open(os.path.join(GOLDEN, "small_dense_seed0.json")) as f:
        g = json.load(f)
    assert hashlib.sha256(got[0].tobytes() + got[1].tobytes()).hexdigest() == g["sha256"]


@pytest.mark.parametrize("kw", [dict(), dict(K=16), dict(K=32), dict(K=8, M=40),
                                dict(r=4), dict(r=5), dict(r=6), dict(y2=1), dict(y2=64), dict(s=1),
                                dict(K=64, y2=4, s=2), dict(K=8, M=62), dict(K=256),
                                dict(y1b=2), dict(y1b=4, s=4), dict(y2=4, y1b=8), dict(K=32, y1b=16)])
def test_plan_invariance(kw):
    """Every valid (K, M, r, tiles) gives byte-identical output."""
    rng = np.random.default_rng(11)
    a = W.random_poly(rng, 300, 255)
    b = W.random_poly(rng, 250, 255)
    check_vs_oracle(a, b, 255, 255, **kw)


# ---- edge cases -------------------------------------------------------------

def test_zero_polynomials():
    a = (np.zeros((10, 2), np.uint32), np.zeros(10, np.uint8))
    b = W.random_poly(np.random.default_rng(1), 7, 50)
    (c, cn), info = gpu_mul(a, b, 50, 50)
    assert not c.any() and not cn.any()


def test_negative_zero_input_and_units():
    a = from_ints([0, -1, 1, 0, -1], 1)
    a[1][0] = 1  # -0
    b = from_ints([1, -1, 0, 1], 1)
    check_vs_oracle(a, b, 1, 1)


def test_single_nonzero_coefficient():
    vals = [0] * 50
    vals[37] = -(1 << 200) + 12345
    a = from_ints(vals, 7)
    b = from_ints([3] + [0] * 20 + [-(1 << 223)], 7)
    check_vs_oracle(a, b, 224, 224)


@pytest.mark.parametrize("na,nb,bits,negative", [(500, 300, 4096, False), (257, 1024, 255, True),
                                                 (1, 64, 1000, True), (4096, 4096, 64, False)])
def test_constant_closed_form(na, nb, bits, negative):
    a = W.constant_poly(na, bits, negative=negative)
    b = W.constant_poly(nb, bits)
    (c, cn), info = gpu_mul(a, b, bits, bits)
    alpha = (1 << bits) - 1
    s = -1 if negative else 1
    want = [s * terms(k, na, nb) * alpha * alpha for k in range(na + nb - 1)]
    assert to_ints(c, cn) == want


@pytest.mark.parametrize("sign_a,sign_b", [(-1, -1), (-1, 1), (1, 1)])
def test_digit_extreme(sign_a, sign_b):
    """Coefficients whose balanced digits are all +-2^(M-1): the products
    c_{i,j} reach the bound H = min(na,nb) K 2^(2M-2) the primes must cover."""
    na = nb = 512
    bits = 1000
    info = ipm.choose(na, nb, bits, bits)
    K, M = info["K"], info["M"]
    J = bits // M  # digits that fit below 2^bits
    half = 1 << (M - 1)
    mag = sum(half << (M * j) for j in range(J))
    assert mag < (1 << bits)
    va = [sign_a * mag] * na
    vb = [sign_b * mag] * nb
    L = W.limbs_for_bits(bits)
    a, b = from_ints(va, L), from_ints(vb, L)
    got, _ = check_vs_oracle(a, b, bits, bits)


def test_bound_violation_is_reported():
    rng = np.random.default_rng(3)
    a = W.random_poly(rng, 16, 40)
    b = W.random_poly(rng, 16, 40)
    a[0][5, 1] |= 1 << 20  # bit 52 set, above the 40-bit bound
    plan = ipm.Plan((16, 16, 40, 40))
    da, dan = ipm.to_device(*a)
    db, dbn = ipm.to_device(*b)
    plan.mul(da, dan, db, dbn)
    with pytest.raises(ipm.IpmError) as e:
        plan.sync()
    assert e.value.status == 2
    # the error word is cleared: a valid call afterwards succeeds
    a[0][5, 1] &= (1 << 8) - 1
    da, dan = ipm.to_device(*a)
    plan.mul(da, dan, db, dbn)
    plan.sync()


def test_batched_with_prebuilt_arguments():
    """mul_batched with the pointer array from batch_args, called twice."""
    shapes = W.batch_shapes(seed=9, count=9, dmin=16, dmax=700, bmin=32, bmax=600)
    ops = W.batch_operands(shapes, seed=9)
    plan = ipm.Plan([(s.na, s.nb, s.bits_a, s.bits_b) for s in shapes])
    dev = [ipm.to_device(*a) + ipm.to_device(*b) for a, b in ops]
    outs = [plan.empty_output(i) for i in range(len(shapes))]
    args = plan.batch_args(dev, outs)
    for _ in range(2):
        for c, cn in outs:
            c.fill_(-1)
            cn.fill_(7)
        assert plan.mul_batched(args) is None
        plan.sync()
        for (a, b), (c, cn), info in zip(ops, outs, plan.infos):
            assert_same(ipm.to_host(c, cn), oracle.polymul(a, b, info["lc"]))
    plan.close()


def test_batched_graph_replay():
    """IPM_GRAPH: the grouped launches are recorded once and replayed; two
    calls on different operand and output buffers (and a product that runs
    outside the graph) all equal the oracle."""
    shapes = W.batch_shapes(seed=12, count=10, dmin=16, dmax=900, bmin=32, bmax=700)
    tuples = [(s.na, s.nb, s.bits_a, s.bits_b) for s in shapes]
    ipm.set_tuned([(tuples[3], {"school": 1})] if tuples[3][0] * tuples[3][1] < 1 << 18 else [])
    try:
        plan = ipm.Plan(tuples, flags=ipm.IPM_GRAPH | ipm.IPM_COSTMODEL)
    finally:
        ipm.set_tuned([])
    for seed in (12, 13):
        ops = W.batch_operands(shapes, seed=seed)
        dev = [ipm.to_device(*a) + ipm.to_device(*b) for a, b in ops]
        outs = plan.mul_batched(dev)
        plan.sync()
        for (a, b), (c, cn), info in zip(ops, outs, plan.infos):
            assert_same(ipm.to_host(c, cn), oracle.polymul(a, b, info["lc"]))
    plan.close()


def test_mul_host_async_two_plans_two_streams():
    """Products in flight on two plans and two streams, host buffers pinned;
    every result equals the oracle's after the syncs."""
    rng = np.random.default_rng(14)
    shape = (600, 500, 300, 200)
    ops = [(W.random_poly(rng, 600, 300), W.random_poly(rng, 500, 200)) for _ in range(4)]
    plans = [ipm.Plan(shape) for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()  # noqa: E731
    I = plans[0].info
    outs = []
    for i, (a, b) in enumerate(ops):
        hc = torch.empty((I["nc"], I["lc"]), dtype=torch.int32).pin_memory().numpy().view(np.uint32)
        hcn = torch.empty((I["nc"],), dtype=torch.uint8).pin_memory().numpy()
        ins = (pin(a[0]), pin(a[1]), pin(b[0]), pin(b[1]))
        plans[i % 2].mul_host_async(*ins, hc, hcn, stream=streams[i % 2])
        outs.append((ins, hc, hcn))
        if i % 2 == 1:  # a plan's buffers are reused by its next call on the same stream
            for pl, st in zip(plans, streams):
                pl.sync(st)
            for (_, hc2, hcn2), (a2, b2) in zip(outs[-2:], ops[i - 1:i + 1]):
                assert_same((hc2, hcn2), oracle.polymul(a2, b2, I["lc"]))
    for pl in plans:
        pl.close()


def test_mul_host_matches_oracle():
    rng = np.random.default_rng(4)
    a = W.random_poly(rng, 700, 500)
    b = W.random_poly(rng, 900, 300)
    plan = ipm.Plan((700, 900, 500, 300))
    c, cn = plan.mul_host(a[0], a[1], b[0], b[1])
    assert_same((c, cn), oracle.polymul(a, b, plan.info["lc"]))
    # second call reuses the staging buffers
    c2, cn2 = plan.mul_host(a[0], a[1], b[0], b[1])
    assert np.array_equal(c, c2) and np.array_equal(cn, cn2)


def test_batched_matches_oracle():
    shapes = W.batch_shapes(seed=3, count=12, dmin=16, dmax=600, bmin=32, bmax=700)
    ops = W.batch_operands(shapes, seed=3)
    plan = ipm.Plan([(s.na, s.nb, s.bits_a, s.bits_b) for s in shapes], flags=ipm.IPM_SYNC)
    dev = []
    for (a, b) in ops:
        da, dan = ipm.to_device(*a)
        db, dbn = ipm.to_device(*b)
        dev.append((da, dan, db, dbn))
    outs = plan.mul_batched(dev)
    torch.cuda.synchronize()
    for s, (a, b), (c, cn), info in zip(shapes, ops, outs, plan.infos):
        assert_same(ipm.to_host(c, cn), oracle.polymul(a, b, info["lc"]))


# ---- full size of the benchmarked workload --------------------------------

def _whole_output_identities(a, b, c):
    A, B, C = to_ints(*a), to_ints(*b), to_ints(*c)
    for t in (1, -1):
        assert eval_at(C, t) == eval_at(A, t) * eval_at(B, t)
    rng = np.random.default_rng(123)
    for q in CHECK_PRIMES:
        t = int(rng.integers(2, 2**60))
        assert oracle.eval_mod(c, t, q) == oracle.eval_mod(a, t, q) * oracle.eval_mod(b, t, q) % q


def assert_full_digest(name, got):
    """Every limb and sign of a full-size product against the oracle's."""
    want = stored_full_digest(name)
    assert want is not None, "tests/golden/full_size_digests.json lacks " + name
    assert full_output_digest(*got) == want


def chosen_plan_params(sh):
    """The parameters the learned dispatch (committed model and sweep
    table, as bench.py installs them) picks for this shape."""
    from paper_1612_05778_gb300 import costmodel as cmod
    cmod.install(points=cmod.load_sweep()["points"])
    prm, _ = ipm.dispatch(sh.na, sh.nb, sh.bits_a, sh.bits_b)
    ipm.set_cost_model(None)
    ipm.set_tuned([])
    return {k: v for k, v in prm.items() if v}


@pytest.mark.parametrize("name,make", [("large_dense", lambda: W.large_dense(seed=1)),
                                       ("huge_dense", lambda: W.huge_dense(seed=2)),
                                       ("huge_mixed", lambda: W.huge_mixed(seed=2))])
def test_full_size_every_limb_with_the_benchmarked_plan(name, make):
    sh, a, b = make()
    got, info = gpu_mul(a, b, sh.bits_a, sh.bits_b, **chosen_plan_params(sh))
    assert info["lc"] == sh.lc
    assert_full_digest(name, got)


def test_large_dense_full_size():
    sh, a, b = W.large_dense(seed=1)
    got, info = gpu_mul(a, b, sh.bits_a, sh.bits_b)
    assert info["lc"] == sh.lc == 257
    assert_full_digest("large_dense", got)
    # sampled coefficients, each computed by the oracle on its own
    nc = sh.nc
    ks = [0, 1, 2, 31, 4095, 16383, 32766, 32767, 32768, 49151, nc - 2, nc - 1]
    ks += np.random.default_rng(5).integers(0, nc, 4).tolist()
    want = oracle.coeffs(ks, a, b, sh.lc)
    assert_same((got[0][ks], got[1][ks]), want)
    _whole_output_identities(a, b, got)


def test_large_all_ones_closed_form():
    sh, a, b = W.large_all_ones()
    (c, cn), info = gpu_mul(a, b, sh.bits_a, sh.bits_b)
    alpha2 = ((1 << 4096) - 1) ** 2
    C = to_ints(c, cn)
    n = sh.na
    bad = [k for k in range(sh.nc) if C[k] != terms(k, n, n) * alpha2]
    assert not bad, bad[:10]


def _sampled_and_identities(sh, a, b, extra_ks=()):
    got, info = gpu_mul(a, b, sh.bits_a, sh.bits_b)
    assert info["lc"] == sh.lc
    nc = sh.nc
    ks = [0, 1, 2, 1000, nc // 4, nc // 2 - 1, nc // 2, nc // 2 + 1, nc - 2, nc - 1, *extra_ks]
    ks += np.random.default_rng(nc).integers(0, nc, 4).tolist()
    want = oracle.coeffs(ks, a, b, sh.lc)
    assert_same((got[0][ks], got[1][ks]), want)
    _whole_output_identities(a, b, got)
    return info, got


def test_huge_dense_full_size():
    """Two degree-262143 polynomials, 1024-bit coefficients (seed 2)."""
    sh, a, b = W.huge_dense(seed=2)
    info, got = _sampled_and_identities(sh, a, b)
    assert info["Y"] == 1 << 19
    assert_full_digest("huge_dense", got)


def test_huge_mixed_full_size():
    """Half the positions < 2^64, the rest < 2^2048, random positions."""
    sh, a, b = W.huge_mixed(seed=2)
    _, got = _sampled_and_identities(sh, a, b)
    assert_full_digest("huge_mixed", got)


def test_batched_with_split_middle_transform():
    """Shapes whose middle transform is split run one by one after the
    grouped launches; the results are the same exact products."""
    shapes = W.batch_shapes(seed=5, count=5, dmin=300, dmax=900, bmin=64, bmax=300)
    ops = W.batch_operands(shapes, seed=5)
    plan = ipm.Plan([(s.na, s.nb, s.bits_a, s.bits_b) for s in shapes], flags=ipm.IPM_SYNC, y1b=2)
    assert all(info["Y1b"] == 2 for info in plan.infos)
    dev = [ipm.to_device(*a) + ipm.to_device(*b) for a, b in ops]
    outs = plan.mul_batched(dev)
    torch.cuda.synchronize()
    for (a, b), (c, cn), info in zip(ops, outs, plan.infos):
        assert_same(ipm.to_host(c, cn), oracle.polymul(a, b, info["lc"]))


def test_naturally_split_wide_product():
    """2^16 coefficients of 16384 bits: the planner splits the middle
    transform (Y2 = 4, Y1 = 32768 = 2048 x 16)."""
    rng = np.random.default_rng(17)
    n, bits = 65536, 16384
    a = W.random_poly(rng, n, bits)
    b = W.random_poly(rng, n, bits)
    got, info = gpu_mul(a, b, bits, bits)
    assert info["Y1b"] > 1
    sh = W.Product(n, n, bits, bits)
    ks = [0, 1, 2, sh.nc - 3, sh.nc - 2, sh.nc - 1]
    want = oracle.coeffs(ks, a, b, sh.lc)
    assert_same((got[0][ks], got[1][ks]), want)
    _whole_output_identities(a, b, got)


# ---- the paper's own table shapes (d = N = 2^k) ----------------------------

@pytest.mark.parametrize("k", [9, 10, 11, 12, 13, 14, 15, 16])
def test_paper_table_shapes(k):
    """Random dense polynomials with degree d equal to the coefficient size N
    (the shapes of the paper's Table classical4andCVL2), seed k: sampled
    coefficients against the oracle where it finishes in seconds (k <= 13),
    and for every k the exact identity c(t) = a(t) b(t) modulo three 61-bit
    primes at random points."""
    d = 1 << k
    rng = np.random.default_rng(k)
    a = W.random_poly(rng, d, d)
    b = W.random_poly(rng, d, d)
    got, info = gpu_mul(a, b, d, d)
    nc = 2 * d - 1
    if k <= 13:
        ks = [0, 1, d - 1, d, nc - 1] + np.random.default_rng(nc).integers(0, nc, 2).tolist()
        assert_same((got[0][ks], got[1][ks]), oracle.coeffs(ks, a, b, info["lc"]))
    rng2 = np.random.default_rng(100 + k)
    for q in CHECK_PRIMES:
        t = int(rng2.integers(2, 2**60))
        assert oracle.eval_mod(got, t, q) == oracle.eval_mod(a, t, q) * oracle.eval_mod(b, t, q) % q


# ---- the supported maxima ------------------------------------------------------

@pytest.mark.parametrize("n,bits", [(1 << 20, 32), (1 << 20, 1024)])
def test_maximum_degree(n, bits):
    """2^20 coefficients per operand: the product's y transform has length
    Y = 2^21, the largest order the primes' roots of unity allow."""
    rng = np.random.default_rng(n + bits)
    a = W.random_poly(rng, n, bits)
    b = W.random_poly(rng, n, bits)
    got, info = gpu_mul(a, b, bits, bits)
    assert info["Y"] == 1 << 21
    nc = 2 * n - 1
    ks = [0, 1, n - 1, n, nc - 2, nc - 1] + np.random.default_rng(nc).integers(0, nc, 2).tolist()
    assert_same((got[0][ks], got[1][ks]), oracle.coeffs(ks, a, b, info["lc"]))
    if bits <= 32:  # C(+-1) = A(+-1) B(+-1) with Python integers (cheap at 32 bits)
        _whole_output_identities(a, b, got)
    rng2 = np.random.default_rng(7)
    for q in CHECK_PRIMES:
        t = int(rng2.integers(2, 2**60))
        assert oracle.eval_mod(got, t, q) == oracle.eval_mod(a, t, q) * oracle.eval_mod(b, t, q) % q


@pytest.mark.parametrize("na,nb,ba,bb", [(4, 3, 65536, 65536), (37, 20, 65536, 1), (1, 1, 65536, 65536)])
def test_maximum_bits(na, nb, ba, bb):
    """Coefficients of the largest supported size (65536 bits): whole
    outputs against the oracle."""
    rng = np.random.default_rng(na * nb)
    a = W.random_poly(rng, na, ba)
    b = W.random_poly(rng, nb, bb)
    check_vs_oracle(a, b, ba, bb)
