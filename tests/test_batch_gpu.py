"""The batched entry point on the full batch workload: 4096 independent
products, degrees and bit bounds log-uniform in [16, 8192] x [32, 4096],
random signs, unbalanced pairs (seed 3), in one ipm_mul_batched call.

Every product is checked by evaluation at a random point modulo the prime
2^61 - 1 (c(t) = a(t) b(t)); a random sample of products is compared limb
by limb with the oracle (whole outputs for the cheap ones, sampled
coefficients for the rest)."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import paper_1612_05778_gb300 as ipm
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
Q = (1 << 61) - 1


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_05778_gb300 import build
    build.build()


@pytest.mark.parametrize("chosen_form", [False, True], ids=["planner", "costmodel_graph"])
def test_full_batch_workload(chosen_form):
    """chosen_form: the flags bench.py times the batch with (the learned
    dispatch with the committed model and sweep table, graph replay)."""
    shapes = W.batch_shapes(seed=3, count=4096)
    ops = W.batch_operands(shapes, seed=3)
    flags = ipm.IPM_SYNC
    if chosen_form:
        from paper_1612_05778_gb300 import costmodel as cmod
        cmod.install(points=cmod.load_sweep()["points"])
        flags |= ipm.IPM_COSTMODEL | ipm.IPM_GRAPH
    plan = ipm.Plan([(s.na, s.nb, s.bits_a, s.bits_b) for s in shapes], flags=flags)
    dev = [ipm.to_device(*a) + ipm.to_device(*b) for a, b in ops]
    outs = [plan.empty_output(i) for i in range(len(shapes))]
    for _ in range(2 if chosen_form else 1):  # a graph is recorded by the first call, replayed by the second
        for c, cn in outs:
            c.fill_(-1)
            cn.fill_(7)
        plan.mul_batched(dev, outs)
    torch.cuda.synchronize()
    host = [ipm.to_host(c, cn) for c, cn in outs]
    rng = np.random.default_rng(31)
    ts = rng.integers(2, Q - 1, len(shapes))

    def check(i):
        (a, b), c, t = ops[i], host[i], int(ts[i])
        return oracle.eval_mod(c, t, Q) == oracle.eval_mod(a, t, Q) * oracle.eval_mod(b, t, Q) % Q

    with ThreadPoolExecutor(max_workers=oracle.default_threads()) as ex:
        ok = list(ex.map(check, range(len(shapes))))
    bad = [i for i, v in enumerate(ok) if not v]
    assert not bad, bad[:10]

    sample = rng.choice(len(shapes), 48, replace=False)
    for i in sample:
        s, (a, b), (c, cn) = shapes[i], ops[i], host[i]
        cost = s.na * s.nb * s.la * s.lb
        if cost < 2e8:
            want = oracle.polymul(a, b, s.lc)
            assert np.array_equal(c, want[0]) and np.array_equal(cn, want[1]), i
        else:
            ks = sorted({0, s.nc - 1, s.nc // 2, *rng.integers(0, s.nc, 5).tolist()})
            want = oracle.coeffs(ks, a, b, s.lc)
            assert np.array_equal(c[ks], want[0]) and np.array_equal(cn[ks], want[1]), i
    plan.close()
    if chosen_form:
        ipm.set_cost_model(None)
        ipm.set_tuned([])
