"""GPU parity for the compile-time instantiated passes on ragged shapes.

The forward, middle and inverse kernels have instantiations whose tile
shape (K, Y2, M for the forward and inverse passes; S, Y1a, K for the middle
pass) is a compile-time constant, chosen at launch when a plan matches.
Inside them, tiles with fewer coefficient rows than the full shape (an
operand shorter than the other, an output shorter than Y) take the
run-time row maps.  These products force plans with those shapes on
unbalanced, ragged operands and compare sampled coefficients with the
oracle limb by limb, plus the exact identities C(1) = A(1)B(1),
C(-1) = A(-1)B(-1) and evaluation modulo three 61-bit primes over the whole
output (integer work: exact equality is the only tolerance).
"""
import numpy as np
import pytest

import oracle
import paper_1612_05778_gb300 as ipm
import workloads as W
from bigint_util import CHECK_PRIMES, eval_at, to_ints

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_05778_gb300 import build
    build.build()


# (na, nb, bits_a, bits_b), plan overrides, the plan fields the
# instantiation is keyed on
CASES = [
    ((200001, 262144, 1024, 1000), dict(K=32, y2=128, s=4),
     dict(K=32, M=33, Y2=128, Y1=4096, S=4)),
    ((30001, 32768, 4096, 3000), dict(K=128, y2=32, s=8),
     dict(K=128, M=33, Y2=32, Y1=2048, S=8)),
    ((131071, 262144, 2048, 1500), dict(K=128, y2=32, s=16),
     dict(K=128, M=17, Y2=32, S=16)),
    # one coefficient against 2^18: every forward tile of a holds at most one row
    ((1, 262144, 1024, 1024), dict(K=32, y2=128, s=4),
     dict(K=32, M=33, Y2=128, S=4)),
]


@pytest.mark.parametrize("shape,params,keys", CASES)
def test_instantiated_shapes_on_ragged_operands(shape, params, keys):
    na, nb, ba, bb = shape
    rng = np.random.default_rng(na + nb)
    a = W.random_poly(rng, na, ba)
    b = W.random_poly(rng, nb, bb)
    plan = ipm.Plan(shape, flags=ipm.IPM_SYNC, **params)
    info = plan.info
    for k, v in keys.items():
        assert info[k] == v, (k, info[k], v)
    da, dan = ipm.to_device(*a)
    db, dbn = ipm.to_device(*b)
    c, cn = plan.mul(da, dan, db, dbn)
    plan.sync()
    got = ipm.to_host(c, cn)
    lc = info["lc"]
    plan.close()
    nc = na + nb - 1
    ks = sorted(k for k in {0, 1, na - 1, na, nb - 1, nb, nc // 2, nc - 2, nc - 1,
                            *rng.integers(0, nc, 5).tolist()} if 0 <= k < nc)
    want = oracle.coeffs(ks, a, b, lc)
    assert np.array_equal(got[0][ks], want[0]) and np.array_equal(got[1][ks], want[1])
    A, B, C = to_ints(*a), to_ints(*b), to_ints(*got)
    for t in (1, -1):
        assert eval_at(C, t) == eval_at(A, t) * eval_at(B, t)
    for q in CHECK_PRIMES:
        t = int(rng.integers(2, 2**60))
        assert oracle.eval_mod(got, t, q) == oracle.eval_mod(a, t, q) * oracle.eval_mod(b, t, q) % q


def test_instantiated_shape_with_a_zero_operand():
    """A zero polynomial times a full one on the bench plan's shape: every
    output limb zero and every sign positive."""
    sh, a, b = W.huge_dense(seed=2)
    a = (np.zeros_like(a[0]), np.ones_like(a[1]))  # -0 everywhere
    plan = ipm.Plan((sh.na, sh.nb, sh.bits_a, sh.bits_b), flags=ipm.IPM_SYNC, K=32, y2=128, s=4)
    assert (plan.info["K"], plan.info["Y2"], plan.info["Y1"], plan.info["S"]) == (32, 128, 4096, 4)
    da, dan = ipm.to_device(*a)
    db, dbn = ipm.to_device(*b)
    c, cn = plan.mul(da, dan, db, dbn)
    plan.sync()
    assert int(c.count_nonzero()) == 0 and int(cn.count_nonzero()) == 0
    plan.close()
