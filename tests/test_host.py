"""Host-side tests (no GPU): the library loads, exports every symbol the
header declares, and the planner (DetermineBase / RecoveryPrime, §2, §2.1,
§4) obeys the paper's conditions."""
import math
import os
import re
import subprocess

import pytest

import paper_1612_05778_gb300 as ipm
from paper_1612_05778_gb300 import build as ipm_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    ipm_build.build()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ipm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ipm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_abi():
    syms = declared_symbols()
    for s in ("ipm_plan", "ipm_mul", "ipm_mul_batched", "ipm_destroy", "ipm_choose", "ipm_mul_host"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    out = subprocess.check_output(["nm", "-D", "--defined-only", ipm.LIB_PATH]).decode()
    exported = set(re.findall(r"\sT\s+(\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_library_loads_without_gpu():
    lib = ipm.load_library()
    assert lib.ipm_strerror(0) == b"ok"
    assert lib.ipm_strerror(2).startswith(b"input coefficient")


SHAPES = [(1, 1, 1, 1), (1024, 1024, 255, 255), (32768, 32768, 4096, 4096), (8192, 16, 4096, 32),
          (262144, 262144, 1024, 1024), (64, 64, 16384, 16384), (3, 700, 33, 7000), (100, 100, 31, 32)]


@pytest.mark.parametrize("shape", SHAPES)
def test_planner_invariants(shape):
    na, nb, ba, bb = shape
    I = ipm.choose(*shape)
    K, M, N, r = I["K"], I["M"], I["N"], I["r"]
    nc = na + nb - 1
    # N = K M with K, M > 1, K a power of two, N >= bits + 1 (two's complement, Eq. definingN)
    assert N == K * M and K >= 2 and M >= 2 and K & (K - 1) == 0
    assert N >= max(ba, bb) + 1
    # y length: power of two >= na + nb - 1 (acyclic product in y)
    Y = I["Y"]
    assert Y & (Y - 1) == 0 and Y >= nc and Y < 2 * max(nc, 1) + 1
    assert I["Y1"] * I["Y2"] == Y
    # every prime has roots of unity of order Y and 2K (Eq. HavingAppropriatePrimitiveRootsOfUnity)
    ps = I["primes"]
    assert len(ps) == r and ps == sorted(ps, reverse=True) and len(set(ps)) == r
    for p in ps:
        assert (1 << 29) < p < (1 << 30)
        assert (p - 1) % max(Y, 2 * K) == 0
    # m = prod p > 4H with H = min(na,nb) * K * 2^(2M-2) (the m > 4H of §1)
    m = math.prod(ps)
    H = min(na, nb) * K * (1 << (2 * M - 2))
    assert m > 4 * H
    # output stride: |c_k| < min(na,nb) 2^(ba+bb) fits in lc limbs
    assert (1 << (32 * I["lc"])) >= min(na, nb) * (1 << (ba + bb))


def test_planner_primes_are_prime():
    sympy = pytest.importorskip("sympy")
    for p in ipm.choose(262144, 262144, 1024, 1024)["primes"] + ipm.choose(64, 64, 16384, 16384)["primes"]:
        assert sympy.isprime(p)


def test_planner_picks_fewest_primes_for_its_split():
    # r is minimal: dropping one prime breaks m > 4H
    for shape in SHAPES:
        I = ipm.choose(*shape)
        if I["r"] == 1:
            continue
        m = math.prod(I["primes"][:-1])
        H = min(shape[0], shape[1]) * I["K"] * (1 << (2 * I["M"] - 2))
        assert m <= 4 * H


@pytest.mark.parametrize("kw", [dict(K=3), dict(K=1), dict(M=1), dict(M=70), dict(r=7),
                                dict(K=8, M=4), dict(r=1, K=8, M=32), dict(y2=3), dict(s=3)])
def test_planner_rejects_invalid_overrides(kw):
    with pytest.raises(ipm.IpmError):
        ipm.choose(1024, 1024, 255, 255, **kw)


@pytest.mark.parametrize("shape", [(0, 5, 8, 8), (5, 5, 0, 8), (5, 5, 8, 70000)])
def test_planner_rejects_bad_shapes(shape):
    with pytest.raises(ipm.IpmError) as e:
        ipm.choose(*shape)
    assert e.value.status == 1


def test_planner_accepts_valid_overrides():
    base = ipm.choose(1024, 1024, 255, 255)
    for kw in (dict(K=16), dict(K=8, M=40), dict(r=4), dict(y2=8), dict(s=2), dict(K=32, y2=1)):
        I = ipm.choose(1024, 1024, 255, 255, **kw)
        for k, v in kw.items():
            key = {"y2": "Y2", "s": "S"}.get(k, k)
            assert I[key] == v
        assert I["lc"] == base["lc"] and I["nc"] == base["nc"]


def test_unsupported_beyond_prime_order():
    # Y would be 2^22 > 2^21, the 2-adic order of every prime
    with pytest.raises(ipm.IpmError) as e:
        ipm.choose(1 << 21, 1 << 21, 64, 64)
    assert e.value.status == 6


# ---- Kronecker balancing plans (host only) ----------------------------------

@pytest.mark.parametrize("shape,s", [((1000, 1000, 32, 32), 2), ((777, 1234, 20, 40), 8),
                                     ((5, 3, 32, 32), 16), ((2048, 2048, 58, 58), 4)])
def test_kron_plan_fields(shape, s):
    na, nb, ba, bb = shape
    info = ipm.choose(*shape, kron=s)
    w = ba + bb + (min(na, nb) - 1).bit_length() + 1
    assert info["kron"] == s and info["kron_w"] == w
    assert info["kron_na"] == -(-na // s) and info["kron_nb"] == -(-nb // s)
    assert info["kron_bits_a"] == ba + (s - 1) * w + 1
    assert info["kron_bits_b"] == bb + (s - 1) * w + 1
    # the output layout is the unpacked product's
    plain = ipm.choose(*shape)
    for k in ("na", "nb", "nc", "la", "lb", "lc"):
        assert info[k] == plain[k]
    assert plain["kron"] == 1 and plain["kron_w"] == 0
    # the inner plan meets the CRT bound of the packed product
    mn = min(info["kron_na"], info["kron_nb"])
    assert info["log2_modulus"] > math.log2(mn) + math.log2(info["K"]) + 2 * info["M"]


@pytest.mark.parametrize("shape,s", [((100, 100, 32, 32), 3), ((100, 100, 32, 32), 32),
                                     ((100, 100, 70, 60), 2), ((100, 100, 32, 32), -1)])
def test_kron_rejects_invalid(shape, s):
    with pytest.raises(ipm.IpmError) as e:
        ipm.choose(*shape, kron=s)
    assert e.value.status == 1


# ---- schoolbook plans (host only) ---------------------------------------------

def test_school_plan_fields():
    info = ipm.choose(300, 257, 255, 255, school=1)
    plain = ipm.choose(300, 257, 255, 255)
    assert info["school"] == 1 and plain["school"] == 0
    for k in ("na", "nb", "nc", "la", "lb", "lc"):
        assert info[k] == plain[k]
    assert info["K"] == info["r"] == info["Y"] == 0
    assert any(c["params"].get("school") for c in ipm.candidates(300, 257, 255, 255))
    assert not any(c["params"].get("school") for c in ipm.candidates(1 << 15, 1 << 15, 4096, 4096))


@pytest.mark.parametrize("shape", SHAPES)
def test_output_limbs_formula_matches_the_planner(shape):
    assert ipm.output_limbs(*shape) == ipm.choose(*shape)["lc"]


def test_plan_free_calls_reject_a_narrow_output_on_the_host():
    """mul_noalloc and validate check c's shape (nc, Lc) before taking any
    pointer or calling the library: a c one limb too narrow would be
    written past its end by the kernels.  CPU tensors suffice, since the
    check comes first."""
    torch = pytest.importorskip("torch")
    na, nb, ba, bb = 300, 200, 255, 100
    lc = ipm.output_limbs(na, nb, ba, bb)
    a = torch.zeros((na, 8), dtype=torch.int32)
    an = torch.zeros((na,), dtype=torch.uint8)
    b = torch.zeros((nb, 4), dtype=torch.int32)
    bn = torch.zeros((nb,), dtype=torch.uint8)
    cn = torch.zeros((na + nb - 1,), dtype=torch.uint8)
    for bad in [(na + nb - 1, lc - 1), (na + nb - 2, lc), (na + nb - 1,)]:
        c = torch.zeros(bad, dtype=torch.int32)
        with pytest.raises(ValueError, match="c must have shape"):
            ipm.mul_noalloc(na, nb, ba, bb, a, an, b, bn, c, cn)
        with pytest.raises(ValueError, match="c must have shape"):
            ipm.validate(na, nb, ba, bb, a, an, b, bn, c, cn)


@pytest.mark.parametrize("shape", [(1, 1, 1, 1), (1024, 1024, 255, 255), (300, 2, 64, 4096), (2048, 2048, 2048, 2048)])
def test_kronecker_substitution_plans(shape):
    """ks=1: slots of w = Lc + 3 limbs; the digit product multiplies
    polynomials of na w and nb w 32-bit coefficients, within the 2^21
    transform length."""
    na, nb, ba, bb = shape
    I = ipm.choose(*shape, ks=1)
    base = ipm.choose(*shape)
    assert I["ks"] == 1 and I["ks_w"] == base["lc"] + 3
    assert (I["na"], I["nb"], I["nc"], I["lc"]) == (na, nb, na + nb - 1, base["lc"])
    w = I["ks_w"]
    assert I["Y"] >= (na + nb) * w - 1 and I["Y"] <= 1 << 21
    assert I["workspace_bytes"] > base["workspace_bytes"] // 4


def test_kronecker_substitution_limits():
    with pytest.raises(ipm.IpmError):
        ipm.choose(4096, 4096, 4096, 4096, ks=1)  # (na + nb) w > 2^21
    with pytest.raises(ipm.IpmError):
        ipm.choose(100, 100, 64, 64, ks=1, kron=2)
    with pytest.raises(ipm.IpmError):
        ipm.choose(100, 100, 64, 64, ks=1, school=1)
    with pytest.raises(ipm.IpmError):
        ipm.choose(100, 100, 64, 64, ks=2)


@pytest.mark.parametrize("levels", [1, 2, 3, 4])
@pytest.mark.parametrize("shape", [(1, 1, 1, 1), (1000, 1000, 255, 255), (700, 1500, 1000, 64), (3, 2000, 64, 64)])
def test_karatsuba_plans(shape, levels):
    """kara=L: operands padded to n2 = m 2^L >= max(na, nb), m < max(na,
    nb) / 2^L + 1; the output layout is the product's own."""
    na, nb, ba, bb = shape
    I = ipm.choose(*shape, kara=levels)
    base = ipm.choose(*shape)
    assert I["kara"] == levels and I["K"] == 0 and I["r"] == 0
    assert (I["na"], I["nb"], I["nc"], I["lc"]) == (na, nb, na + nb - 1, base["lc"])
    assert I["workspace_bytes"] > 0


def test_karatsuba_limits():
    with pytest.raises(ipm.IpmError):
        ipm.choose(100, 100, 64, 64, kara=5)
    with pytest.raises(ipm.IpmError):
        ipm.choose(100, 100, 64, 64, kara=2, K=8)
    with pytest.raises(ipm.IpmError):
        ipm.choose(100, 100, 8192, 8192, kara=1)  # leaf columns beyond the schoolbook kernel's


@pytest.mark.parametrize("shape", [(1, 1, 1, 1), (1024, 1024, 255, 255), (2048, 2048, 2048, 2048), (5, 9, 4096, 4096)])
def test_big_prime_plans(shape):
    """bigp=1: one prime p = (2^63 + 2^53)^2 + 1 (log2 p = 126.003), the
    smallest K with N = K M >= bits + 1, M <= 62 and 4H < p."""
    na, nb, ba, bb = shape
    I = ipm.choose(*shape, bigp=1)
    K, M = I["K"], I["M"]
    mn = min(na, nb)
    assert I["bigp"] == 1 and I["r"] == 1 and K * M == I["N"] >= max(ba, bb) + 1 and M <= 62
    assert 4 * mn * K * 2 ** (2 * M - 2) < (2**63 + 2**53) ** 2 + 1
    if K > 2:  # a smaller K would break the bound or M <= 62
        k2 = K // 2
        m2 = max(2, -(-(max(ba, bb) + 1) // k2))
        assert m2 > 62 or 4 * mn * k2 * 2 ** (2 * m2 - 2) >= (2**63 + 2**53) ** 2 + 1


def test_big_prime_limits():
    with pytest.raises(ipm.IpmError):
        ipm.choose(100, 100, 64, 64, bigp=1, r=2)
    with pytest.raises(ipm.IpmError):
        ipm.choose(100, 100, 64, 64, bigp=2)
