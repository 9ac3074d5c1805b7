"""Batched calls as one persistent launch over a device work queue
(IPM_PERSISTENT): every product of the queue against the oracle, with and
without graph replay, schoolbook products inside the queue, the full
4096-product batch, and the timeout path -- a product whose forward phase
is held open (a counter nothing completes) makes its later tiles' bounded
waits run out, the call reports IPM_ERR_TIMEOUT, and the same plan then
computes correct products again (nothing faults or hangs the GPU)."""
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


def run_batch(shapes, ops, flags, calls=1, **kw):
    plan = ipm.Plan([(s.na, s.nb, s.bits_a, s.bits_b) for s in shapes], flags=flags | ipm.IPM_PERSISTENT, **kw)
    dev = [ipm.to_device(*a) + ipm.to_device(*b) for a, b in ops]
    outs = [plan.empty_output(i) for i in range(len(shapes))]
    for _ in range(calls):
        for c, cn in outs:
            c.fill_(-1)
            cn.fill_(7)
        plan.mul_batched(dev, outs)
        plan.sync()
    host = [ipm.to_host(c, cn) for c, cn in outs]
    return plan, dev, outs, host


def check_all(shapes, ops, host, full_limit=2e8):
    rng = np.random.default_rng(77)
    for s, (a, b), (c, cn) in zip(shapes, ops, host):
        if s.na * s.nb * s.la * s.lb < full_limit:
            want = oracle.polymul(a, b, s.lc)
            assert np.array_equal(c, want[0]) and np.array_equal(cn, want[1]), (s.na, s.nb, s.bits_a, s.bits_b)
        else:
            ks = sorted({0, s.nc - 1, s.nc // 2, *rng.integers(0, s.nc, 4).tolist()})
            want = oracle.coeffs(ks, a, b, s.lc)
            assert np.array_equal(c[ks], want[0]) and np.array_equal(cn[ks], want[1])


@pytest.mark.parametrize("graph", [False, True])
def test_queue_matches_the_oracle(graph):
    shapes = W.batch_shapes(seed=21, count=60, dmin=16, dmax=3000, bmin=32, bmax=2000)
    ops = W.batch_operands(shapes, seed=21)
    plan, _, _, host = run_batch(shapes, ops, ipm.IPM_SYNC | (ipm.IPM_GRAPH if graph else 0), calls=2)
    check_all(shapes, ops, host)
    plan.close()


def test_schoolbook_products_in_the_queue():
    shapes = W.batch_shapes(seed=22, count=30, dmin=2, dmax=200, bmin=8, bmax=900)
    ops = W.batch_operands(shapes, seed=22)
    plan, _, _, host = run_batch(shapes, ops, ipm.IPM_SYNC, school=1)
    assert all(i["school"] for i in plan.infos)
    check_all(shapes, ops, host)
    plan.close()


def test_full_batch_workload_with_the_bench_flags():
    from paper_1612_05778_gb300 import costmodel as cmod
    cmod.install(points=cmod.load_sweep()["points"])
    shapes = W.batch_shapes(seed=3, count=4096)
    ops = W.batch_operands(shapes, seed=3)
    plan, _, _, host = run_batch(shapes, ops, ipm.IPM_SYNC | ipm.IPM_COSTMODEL | ipm.IPM_GRAPH, calls=2)
    ipm.set_cost_model(None)
    ipm.set_tuned([])
    ts = np.random.default_rng(31).integers(2, Q - 1, len(shapes))

    def check(i):
        (a, b), c, t = ops[i], host[i], int(ts[i])
        return oracle.eval_mod(c, t, Q) == oracle.eval_mod(a, t, Q) * oracle.eval_mod(b, t, Q) % Q

    with ThreadPoolExecutor(max_workers=oracle.default_threads()) as ex:
        ok = list(ex.map(check, range(len(shapes))))
    assert all(ok), [i for i, v in enumerate(ok) if not v][:10]
    sample = np.random.default_rng(5).choice(len(shapes), 24, replace=False)
    check_all([shapes[i] for i in sample], [ops[i] for i in sample], [host[i] for i in sample])
    plan.close()


def test_a_wait_that_runs_out_reports_a_timeout_and_the_plan_recovers():
    shapes = W.batch_shapes(seed=23, count=12, dmin=100, dmax=2000, bmin=64, bmax=1000)
    ops = W.batch_operands(shapes, seed=23)
    plan = ipm.Plan([(s.na, s.nb, s.bits_a, s.bits_b) for s in shapes], flags=ipm.IPM_PERSISTENT)
    dev = [ipm.to_device(*a) + ipm.to_device(*b) for a, b in ops]
    outs = [plan.empty_output(i) for i in range(len(shapes))]
    plan.set_wait_limit(20000)  # 20 ms
    plan.debug_hold(3)          # product 3's forward phase can never complete
    plan.mul_batched(dev, outs)
    with pytest.raises(ipm.IpmError) as e:
        plan.sync()
    assert e.value.status == 5  # IPM_ERR_TIMEOUT
    plan.debug_hold(-1)
    plan.set_wait_limit(2000000)
    plan.mul_batched(dev, outs)
    plan.sync()
    check_all(shapes, ops, [ipm.to_host(c, cn) for c, cn in outs])
    plan.close()


def test_controls_need_a_persistent_plan():
    plan = ipm.Plan([(100, 100, 64, 64), (50, 70, 32, 32)])
    with pytest.raises(ipm.IpmError) as e:
        plan.set_wait_limit(1000)
    assert e.value.status == 6  # IPM_ERR_UNSUPPORTED
    plan.close()
