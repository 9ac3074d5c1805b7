"""ipm_mul_noalloc: the product entry point that allocates nothing.

It serves callers that may not allocate device memory while they run
(services that forbid allocator calls because cudaMalloc can synchronise
the device, plugins whose host application owns all memory).  Its scratch is one static device
array shared by all calls, so this checks two calls in a row -- the second
sees the first call's leftovers in the array -- against ipm_mul, the
allocating entry point, bit for bit (the tolerance of every integer test
here).  The file is named to be collected last.
"""
import numpy as np
import pytest

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


def _product_with_plan(shape, a, b):
    plan = ipm.Plan(shape, flags=ipm.IPM_SYNC)
    da, dan = ipm.to_device(*a)
    db, dbn = ipm.to_device(*b)
    c, cn = plan.mul(da, dan, db, dbn)
    torch.cuda.synchronize()
    out = ipm.to_host(c, cn)
    lc = plan.info["lc"]
    plan.close()
    return out, lc


def _product_noalloc(shape, a, b, lc):
    na, nb, ba, bb = shape
    da, dan = ipm.to_device(*a)
    db, dbn = ipm.to_device(*b)
    # output buffers filled with garbage: every limb must be written
    c = torch.full((na + nb - 1, lc), -1, dtype=torch.int32, device="cuda")
    cn = torch.full((na + nb - 1,), 7, dtype=torch.uint8, device="cuda")
    ipm.mul_noalloc(na, nb, ba, bb, da, dan, db, dbn, c, cn)
    return ipm.to_host(c, cn)


def test_two_calls_in_a_row_match_ipm_mul():
    rng = np.random.default_rng(2024)
    # call 1: the small dense shape; call 2: a different shape, so the second
    # call runs over the first call's tables and workspace left in the array
    for shape in [(1024, 1024, 255, 255), (700, 1500, 1000, 64)]:
        na, nb, ba, bb = shape
        a = W.random_poly(rng, na, ba)
        b = W.random_poly(rng, nb, bb)
        want, lc = _product_with_plan(shape, a, b)
        got = _product_noalloc(shape, a, b, lc)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), shape


def test_same_shape_twice_with_new_inputs():
    rng = np.random.default_rng(7)
    shape = (513, 257, 300, 300)
    for _ in range(2):
        a = W.random_poly(rng, shape[0], shape[2])
        b = W.random_poly(rng, shape[1], shape[3])
        want, lc = _product_with_plan(shape, a, b)
        got = _product_noalloc(shape, a, b, lc)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_rejects_products_larger_than_the_scratch():
    na = nb = 4096
    bits = 4096  # needs 48.4 MiB of scratch > 32 MiB
    a = (torch.zeros((na, 128), dtype=torch.int32, device="cuda"),
         torch.zeros((na,), dtype=torch.uint8, device="cuda"))
    c = torch.zeros((2 * na - 1, 257), dtype=torch.int32, device="cuda")
    cn = torch.zeros((2 * na - 1,), dtype=torch.uint8, device="cuda")
    with pytest.raises(ipm.IpmError) as e:
        ipm.mul_noalloc(na, nb, bits, bits, a[0], a[1], a[0], a[1], c, cn)
    assert e.value.status == 6  # IPM_ERR_UNSUPPORTED, found on the host
