"""Benchmark: exact dense Z[y] products on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload huge_dense|large_dense|small_dense|large_all_ones|huge_mixed|batch|taylor|paper_table|families]

One step is one whole product c = a*b (split, forward 2-D transforms over
every prime, pointwise products, inverse transforms, CRT, recombination)
through the C ABI, by default on the largest one-GPU workload: two
polynomials of degree 262143 with 1024-bit signed coefficients (seed 2).
Inputs are resident in HBM before the timed region; the L2 is flushed (a
512 MiB write) between timed steps, outside the events.  Prints ONE JSON
line on rank 0.  The same line carries, under `extras`, the product of two
degree-32767 polynomials with 4096-bit coefficients (seed 1), the mixed
variant of the default workload (half the coefficients below 2^64, the rest
below 2^2048) and the 4096-product batch with its speedup over the plain
path (--no-extras skips them).

--impl reference times the CPU oracle (plain schoolbook definition, all
host cores) on a bounded sample of the same workload per step and
extrapolates to products/s.

The timed plan is the one the learned dispatch picks (IPM_COSTMODEL with
the committed GB300 cost model and the sweep's table of measured bests,
which takes precedence for shapes the sweep timed); `--plain` times the
analytic planner's plan instead.  When the two differ, the plain plan is timed beside it on the
same inputs and `speedup_vs_plain` is the ratio (1 when they coincide).

--workload batch times one ipm_mul_batched call over 4096 products of
log-uniform degrees in [16, 8192] and bit bounds in [32, 4096] (seed 3) with
the learned dispatch, its grouped launches replayed as one CUDA graph, and,
beside it, the same batch with the analytic planner and the same products
as 4096 ipm_mul calls (the plain path);
`speedup_vs_plain` is the ratio to the plain path.

--workload paper_table times the shapes of the paper's own table (d = N =
2^9 .. 2^16) and lists the paper's 48-core CVL_p^2 seconds beside each row.

--workload families times every product family (learned dispatch, 2-D
transform, schoolbook, Karatsuba with 1..4 levels, Kronecker substitution,
the big-prime form) on a grid of balanced shapes.

--workload taylor times ipm_taylor_shift, g(x) = f(x + 1), on 2^14
coefficients below 2^4096 (seed 5), and prints its own line (shifts/s).

Every default run also times the same product with the tensor-core radix-16
stages (IPM_TENSOR_STAGES; `tensor_stages` in the line, --no-tensor skips it).

Multi-GPU (torchrun): products are independent, so every rank multiplies its
own pair (weak scaling, no data-path collective); the host-side barrier and
max-over-ranks timing use torch.distributed.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "exact Z[x] products/s and output Gbit/s at (d,N); speedup vs plain GPU path"
UNIT = "products/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
PASS_NAMES = ["k_forward", "k_middle", "k_inverse"]
E2E_INFLIGHT = 3  # products in flight in the end-to-end measurement
KERNEL_SRC = [os.path.join(ROOT, "paper_1612_05778_gb300", "csrc", n)
              for n in ("ipm_kernels.cu", "passes.cuh", "ntt_stages.cuh", "modarith.cuh", "ipm_internal.h")]
DEFAULT_WORKLOAD = "huge_dense"


def workload(name: str):
    if name == "large_dense":
        sh, a, b = W.large_dense(seed=1)
        return "large_dense: d=32768, |coeff| < 2^4096, signed uniform, seed 1", sh, a, b
    if name == "small_dense":
        sh, a, b = W.small_dense(seed=0)
        return "small_dense: d=1024, |coeff| < 2^255, signed uniform, seed 0", sh, a, b
    if name == "large_all_ones":
        sh, a, b = W.large_all_ones()
        return "large_all_ones: d=32768, every coefficient 2^4096-1", sh, a, b
    if name == "huge_dense":
        sh, a, b = W.huge_dense(seed=2)
        return "huge_dense: d=262144, |coeff| < 2^1024, signed uniform, seed 2", sh, a, b
    if name == "huge_mixed":
        sh, a, b = W.huge_mixed(seed=2)
        return ("huge_mixed: d=262144, half the positions < 2^64, the rest < 2^2048, signed, seed 2", sh, a, b)
    raise SystemExit("unknown workload " + name)


def workload_config(name, sh):
    """The `config` of both arms' JSON lines: the workload alone."""
    return {"workload": name, "na": sh.na, "nb": sh.nb, "bits": sh.bits_a, "lc": sh.lc}


# ---------------------------------------------------------------------------
# distributed plumbing (host side only)
# ---------------------------------------------------------------------------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def max_over_ranks(dist, value: float, device=None) -> float:
    """Largest value over all ranks (host-side timing reduction)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3] not in ("", "[N/A]"))}


# ---------------------------------------------------------------------------
# oracle (CPU) timing: a bounded sample of output coefficients
# ---------------------------------------------------------------------------

def oracle_sample_time(sh, a, b, target_s: float, seed: int = 0):
    """Time the oracle on sampled output coefficients and extrapolate to a
    full product: a coefficient c_k costs terms(k) limb products of the two
    operand rows, the whole product costs na*nb of them."""
    import oracle
    threads = oracle.default_threads()
    rng = np.random.default_rng(seed)

    def terms(k):
        return max(0, min(k, sh.na - 1) - max(0, k - (sh.nb - 1)) + 1)

    def run(count):
        ks = np.sort(rng.integers(0, sh.nc, count))
        t0 = time.perf_counter()
        oracle.coeffs(ks, a, b, sh.lc, threads=threads)
        dt = time.perf_counter() - t0
        work = sum(terms(int(k)) for k in ks)
        return dt, work, count

    dt, work, count = run(max(threads, 8))
    if dt < target_s * 0.5:
        want = int(count * target_s / max(dt, 1e-3))
        want = max(count, min(want, sh.nc))
        dt, work, count = run(want)
    full = float(sh.na) * float(sh.nb)
    t_full = dt * full / max(work, 1)
    return {"products_per_s": 1.0 / t_full, "seconds": dt, "coefficients": count,
            "fraction_of_product": work / full, "threads": threads}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    name, sh, a, b = workload(args.workload)
    import oracle
    oracle.build()
    per_step = max(1.0, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample_time(sh, a, b, per_step * 0.3, seed=100)
    vals = []
    secs = 0.0
    last = None
    for s in range(args.steps):
        r = oracle_sample_time(sh, a, b, per_step, seed=s)
        vals.append(r["products_per_s"])
        secs += r["seconds"]
        last = r
    value = float(np.median(vals))
    out_bits = sh.nc * sh.lc * 32
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "output_gbit_s": out_bits * value / 1e9,
        "config": workload_config(name, sh),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["threads"], "kind": "oracle",
                         "sample": "per step: %d random output coefficients (%.3g%% of the product's "
                                   "limb products), timed and scaled to one whole product"
                                   % (last["coefficients"], 100 * last["fraction_of_product"])},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def io_bytes(info):
    """Bytes of the operands (limbs and sign bytes) and of the output."""
    inp = info["na"] * (info["la"] * 4 + 1) + info["nb"] * (info["lb"] * 4 + 1)
    out = info["nc"] * (info["lc"] * 4 + 1)
    return inp, out


def algorithmic_bytes(info):
    """DRAM bytes each pass of this implementation moves for one product:
    forward reads both operands and writes 2 r Y 2K residues (both x halves
    of both operands); middle reads them and writes r Y 2K; inverse reads r
    Y 2K and writes the output.  With R = r Y K 4 bytes: in + 4R, 6R,
    2R + out (in + out + 12R in all)."""
    z = info["r"] * info["Y"] * 2 * info["K"] * 4
    inp, out = io_bytes(info)
    return [inp + 2 * z, 3 * z, z + out]


def schedule_bytes(info):
    """The three-pass byte count of the method's minimal schedule, R = r Y K
    4 bytes: forward writes 2R (one K-column slab per operand), middle
    reads 2R and writes 2R (the product's two x halves), inverse reads 2R:
    in + 2R, 4R, 2R + out (in + out + 8R in all)."""
    R = info["r"] * info["Y"] * info["K"] * 4
    inp, out = io_bytes(info)
    return [inp + 2 * R, 4 * R, 2 * R + out]


# 32-bit integer instructions per algorithmic unit: a lazy
# Shoup butterfly (3 multiplies, 2 additions, 1 conditional subtraction and
# the twiddle's subtraction) 7, a Shoup multiplication by a constant 3, a
# Montgomery product 5.
OPS_BUTTERFLY, OPS_SHOUP, OPS_MONT = 7, 3, 5


def algorithmic_int_ops(info):
    """Algorithmic 32-bit integer operations of each pass for one product:
    radix-2 butterflies of every transform, constant multiplications
    (residues, twist, four-step twiddles, untwist, CRT) and pointwise
    Montgomery products, weighted as above."""
    r, Y, K = info["r"], info["Y"], info["K"]
    n_in = info["na"] + info["nb"]
    lgK = max(0, K.bit_length() - 1)
    lgY1 = max(0, info["Y1"].bit_length() - 1)
    lgY2 = max(0, info["Y2"].bit_length() - 1)
    # forward: x-DFTs of the rows holding coefficients, y step A, twist,
    # residues (2 multiplies per digit), step-B twiddle
    bf_f = r * n_in * K * lgK + 2 * r * Y * K * lgY2
    mul_f = r * n_in * K * 3 + 2 * r * Y * 2 * K
    # middle: y step C for A and B, pointwise product, inverse step C
    bf_m = 3 * r * Y * K * lgY1
    mont_m = r * Y * 2 * K
    # inverse: y step A, x-DFTs of the output rows, step-B twiddle, untwist
    # (2 multiplies per pair), Garner (r(r-1)/2 multiplies per value)
    nc = info["nc"]
    bf_i = r * Y * K * lgY2 + r * nc * K * lgK
    mul_i = r * Y * 2 * K + 2 * r * nc * K + (r * (r - 1) // 2) * nc * 2 * K
    return [OPS_BUTTERFLY * bf_f + OPS_SHOUP * mul_f,
            OPS_BUTTERFLY * bf_m + OPS_MONT * mont_m,
            OPS_BUTTERFLY * bf_i + OPS_SHOUP * mul_i]


def stage_bits(logL: int):
    """Radix exponents of the register stages of a length-2^logL transform
    (at most 4 bits each, as even as possible, larger first)."""
    nst = (logL + 3) // 4
    if nst == 0:
        return []
    base, extra = logL // nst, logL % nst
    return [base + (1 if i < extra else 0) for i in range(nst)]


# INT8 mma.sync m16n8k32 throughput on a GB300, measured with a
# microbenchmark (1216 blocks x 128 threads, eight independent accumulator
# chains per warp, operands in registers): 151.0 Tops/s.  tcgen05.mma has no
# 8-bit integer kind on sm_103a (ptxas rejects .kind::i8 for that target).
INT8_MMA_SYNC_TOPS = 151.0


def tensor_stage_ops(info, na: int, nb: int):
    """INT8 tensor operations (2 per multiply-add) of the radix-16 stages of
    one product under IPM_TENSOR_STAGES, per pass [forward (+outer),
    middle, inverse (+outer)]: a stage vector of 16 elements costs 4 byte
    slices x 2 K-chunks of 16 x 8 x 32 products shared by 8 vectors, i.e.
    8192 operations (4096 when its upper half is zero)."""
    r, Y, K = info["r"], info["Y"], info["K"]
    Y1, Y2, Y1b = info["Y1"], info["Y2"], info["Y1b"]
    lg = lambda x: int(x).bit_length() - 1  # noqa: E731
    n16 = lambda logL: sum(1 for b in stage_bits(logL) if b == 4)  # noqa: E731
    full = 8192
    fwd = 0
    for n in (na, nb):
        fwd += n16(lg(K)) * (n * 2 * K // 16) * full          # x DFTs of the coefficient rows
        sb = stage_bits(lg(Y2))
        if sb:
            i1 = np.arange(Y1)
            nr = np.clip((n - i1 + Y1 - 1) // Y1, 0, Y2)
            hz = int(np.count_nonzero((Y2 >= 2) & (2 * nr <= Y2)))
            per_tile = Y2 * 2 * K // 16
            for i, b in enumerate(sb):
                if b == 4:
                    cost = hz * 4096 + (Y1 - hz) * full if i == 0 else Y1 * full
                    fwd += per_tile * cost
    mid_bits = stage_bits(lg(Y1 // Y1b))
    mid = 0
    if len(mid_bits) >= 2:
        k16 = sum(1 for b in mid_bits[:-1] if b == 4)
        mid = 3 * k16 * (Y * 2 * K // 16) * full                # A and B forward, the product inverse
    outer = n16(lg(Y1b)) * (Y * 2 * K // 16) * full if Y1b > 1 else 0
    inv = n16(lg(Y2)) * (Y * 2 * K // 16) * full + n16(lg(K)) * (info["nc"] * 2 * K // 16) * full
    return [r * (fwd + 2 * outer), r * mid, r * (inv + outer)]


def alu_peak_tops(sm_mhz_max: float) -> float:
    """Integer issue peak: 152 SMs x 4 schedulers x 32 lanes, one 32-bit
    instruction per lane per cycle, at the maximum SM clock."""
    return 152 * 4 * 32 * sm_mhz_max * 1e6 / 1e12


def load_peak_hbm():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    """Hash of the sources the three pass kernels are compiled from."""
    h = hashlib.sha256()
    for path in KERNEL_SRC:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload_name: str):
    """DRAM bytes per launch of `kernel` on `workload_name` from the
    committed ncu summary profiles/traffic_<workload>.md, or None when the
    summary is missing or was taken on other kernel source."""
    try:
        text = open(os.path.join(ROOT, "profiles", "traffic_%s.md" % workload_name)).read()
    except OSError:
        return None
    m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    if not m or m.group(1) != kernel_source_hash():
        return None
    m = re.search(r"^%s_dram_bytes_per_launch:\s*([0-9]+)" % kernel, text, re.M)
    return int(m.group(1)) if m else None


BATCH_WORKLOAD = ("batch: 4096 products, degrees log-uniform in [16, 8192], bits log-uniform in [32, 4096], "
                  "random signs, unbalanced pairs, seed 3")


def timed_ms(torch, fn, steps, flush, stream):
    """Mean event-timed duration of fn() on `stream` over `steps` calls, the
    L2 flushed (a 512 MiB write) before each call, outside the events."""
    ms = []
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return float(np.mean(ms))


def measure_batch(ipm, torch, steps, warmup, plain_path, flush, rank=0, world=1, dist=None):
    """One ipm_mul_batched call over the 4096-product batch (seed 3): the
    chosen form (learned dispatch + graph replay; the analytic planner with
    plain_path) against the same batch with the analytic planner and the
    same products as 4096 ipm_mul calls (the plain path).  With world > 1
    every rank runs its own share of the products (paper_1612_05778_gb300.
    shard: cost-balanced, no data-path collective) and the times are the
    maximum over ranks."""
    from paper_1612_05778_gb300 import shard
    all_shapes = W.batch_shapes(seed=3, count=4096)
    all_ops = W.batch_operands(all_shapes, seed=3)
    mine = list(range(len(all_shapes)))
    split = None
    if world > 1:
        costs = shard.shape_costs([(s.na, s.nb, s.bits_a, s.bits_b) for s in all_shapes])
        parts = shard.partition(costs, world)
        mine = parts[rank]
        ld = shard.loads(costs, parts)
        split = {"ranks": world, "products_per_rank": [len(p) for p in parts],
                 "cost_imbalance": max(ld) / (sum(ld) / world)}
    shapes = [all_shapes[i] for i in mine]
    ops = [all_ops[i] for i in mine]
    tuples = [(s.na, s.nb, s.bits_a, s.bits_b) for s in shapes]
    flags = 0
    if not plain_path:
        from paper_1612_05778_gb300 import costmodel as cmod
        cmod.install(points=cmod.load_sweep()["points"])  # model + the sweep's table
        flags = ipm.IPM_COSTMODEL | ipm.IPM_GRAPH
    plan = ipm.Plan(tuples, flags=flags)            # the chosen form
    plan_planner = ipm.Plan(tuples)                 # batched, analytic planner
    plan_persist = ipm.Plan(tuples, flags=flags | ipm.IPM_PERSISTENT)  # one persistent launch
    dev = [ipm.to_device(*a) + ipm.to_device(*b) for a, b in ops]
    outs = [plan.empty_output(i) for i in range(len(shapes))]
    singles = [ipm.Plan((s.na, s.nb, s.bits_a, s.bits_b)) for s in shapes]
    stream = torch.cuda.current_stream()
    # the timed region holds the C ABI calls; the binding's argument checks
    # and pointer tables are prepared before it (ipm_mul_batched still copies
    # its pointer table to the device on every call)
    bargs = plan.batch_args(dev, outs)
    bargs_planner = plan_planner.batch_args(dev, outs)
    outs_p = [plan_persist.empty_output(i) for i in range(len(shapes))]
    bargs_persist = plan_persist.batch_args(dev, outs_p)
    batched = lambda: plan.mul_batched(bargs, stream=stream)  # noqa: E731
    batched_planner = lambda: plan_planner.mul_batched(bargs_planner, stream=stream)  # noqa: E731
    batched_persist = lambda: plan_persist.mul_batched(bargs_persist, stream=stream)  # noqa: E731
    lib = ipm.load_library()
    sh = ctypes.c_void_p(int(stream.cuda_stream))
    calls = [(sp._h,) + tuple(ctypes.c_void_p(t.data_ptr()) for t in (da, dan, db, dbn, c, cn))
             for sp, (da, dan, db, dbn), (c, cn) in zip(singles, dev, outs)]

    def plain():
        for h, *ptrs in calls:
            st = lib.ipm_mul(h, *ptrs, sh)
            if st:
                raise SystemExit("ipm_mul failed: %d" % st)

    for _ in range(warmup):
        batched()
        batched_planner()
        batched_persist()
        plain()
    torch.cuda.synchronize()
    plan.sync()
    plan_planner.sync()
    l0 = ipm.launch_count()
    barrier(dist)
    ms_b = max_over_ranks(dist, timed_ms(torch, batched, steps, flush, stream), torch.cuda.current_device())
    launches = ipm.launch_count() - l0
    ms_bp = max_over_ranks(dist, timed_ms(torch, batched_planner, max(1, steps // 2), flush, stream),
                           torch.cuda.current_device())
    ms_p = max_over_ranks(dist, timed_ms(torch, plain, max(1, steps // 2), flush, stream),
                          torch.cuda.current_device())
    ms_pp = max_over_ranks(dist, timed_ms(torch, batched_persist, max(1, steps // 2), flush, stream),
                           torch.cuda.current_device())
    plan_planner.sync()
    plan.sync()
    plan_persist.sync()
    same_p = all(torch.equal(x[0], y[0]) and torch.equal(x[1], y[1]) for x, y in zip(outs, outs_p))
    if not same_p:
        raise SystemExit("the persistent launch and the grouped launches disagree")
    changed = sum(any(a[k] != b[k] for k in ("K", "M", "r", "Y2", "S", "Y1b", "kron", "school"))
                  for a, b in zip(plan.infos, plan_planner.infos))
    n = len(all_shapes)
    out_bits = sum(s.nc * s.lc * 32 for s in all_shapes)
    res = {"value": n / (ms_b / 1e3), "unit": UNIT, "ms_per_batch": ms_b, "products": n,
           "output_gbit_s": out_bits / (ms_b / 1e3) / 1e9, "speedup_vs_plain": ms_p / ms_b,
           "plain": {"ms_per_batch": ms_p, "value": n / (ms_p / 1e3),
                     "path": "one ipm_mul C call per product (pointers prepared), analytic planner"},
           "batched_planner": {"ms_per_batch": ms_bp, "value": n / (ms_bp / 1e3),
                               "path": "one ipm_mul_batched call, analytic planner"},
           "persistent": {"ms_per_batch": ms_pp, "value": n / (ms_pp / 1e3),
                          "path": "the chosen form's plans as ONE persistent launch over a device work queue "
                                  "(IPM_PERSISTENT, graph-replayed); outputs byte-identical"},
           "dispatch": {"flags": "IPM_COSTMODEL | IPM_GRAPH" if flags else "none (--plain)",
                        "products_with_another_plan": int(changed)},
           "workload": BATCH_WORKLOAD, "gpu_launches": int(launches), "launches_per_call": launches / steps,
           "split": split}
    for sp in singles:
        sp.close()
    plan.close()
    plan_planner.close()
    plan_persist.close()
    return res


def run_batch(args):
    """The batched workload alone: products/s of one ipm_mul_batched call
    (and of the same products one ipm_mul at a time).  Under torchrun the
    4096 products are split across the ranks (strong scaling: the total
    work is fixed)."""
    import torch
    world, rank, local = dist_env()
    dist = dist_init(world, "nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1612_05778_gb300 import build as ipm_build
    if rank == 0:
        ipm_build.build()
    barrier(dist)
    import paper_1612_05778_gb300 as ipm
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    r = measure_batch(ipm, torch, args.steps, args.warmup, args.plain, flush, rank, world, dist)
    clocks = sampler.stop()
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_batch"], "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "split": r["split"],
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "output_gbit_s": r["output_gbit_s"], "speedup_vs_plain": r["speedup_vs_plain"],
            "plain": r["plain"], "batched_planner": r["batched_planner"], "persistent": r["persistent"],
            "dispatch": r["dispatch"],
            "config": {"workload": BATCH_WORKLOAD},
            "setup": {"products": r["products"], "l2": "flushed between timed steps"},
            "gpu_launches": r["gpu_launches"], "launches_per_step": r["launches_per_call"], "clocks": clocks}
    print(json.dumps(line))
    return 0


def run_taylor(args):
    """Taylor shift by one, g(x) = f(x + 1), of 2^14 coefficients below
    2^4096 (seed 5) through ipm_taylor_shift: shifts/s, inputs resident on
    the device, L2 flushed between timed steps; the oracle's sampled
    coefficients (g_k = sum_{i>=k} C(i,k) f_i, Python integers, one core)
    scaled to a whole shift as the CPU baseline."""
    import torch
    torch.cuda.set_device(0)
    from paper_1612_05778_gb300 import build as ipm_build
    ipm_build.build()
    import paper_1612_05778_gb300 as ipm
    (n, bits), f = W.taylor_dense(seed=5)
    # the level products take the plans the learned dispatch picks
    from paper_1612_05778_gb300 import costmodel as cmod
    cmod.install(points=cmod.load_sweep()["points"])
    ts = ipm.TaylorShift(n, bits, flags=ipm.IPM_COSTMODEL)
    df, dfn = ipm.to_device(*f)
    g = torch.empty((n, ts.limbs), dtype=torch.int32, device="cuda")
    gn = torch.empty((n,), dtype=torch.uint8, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ts.shift(df, dfn, g, gn)
    ts.sync()
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    l0 = ipm.launch_count()
    ms = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ts.shift(df, dfn, g, gn, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    launches = ipm.launch_count() - l0
    clocks = sampler.stop()
    ts.sync()
    t_ms = float(np.mean(ms))
    cpu = None
    if not args.no_cpu_baseline:
        from oracle.taylor import taylor_coeff
        F = [(-1 if s else 1) * int.from_bytes(row.tobytes(), "little") for row, s in zip(f[0], f[1])]
        rng = np.random.default_rng(0)
        done, work, t0 = 0, 0, time.perf_counter()
        while time.perf_counter() - t0 < args.cpu_seconds:
            k = int(rng.integers(0, n))
            taylor_coeff(F, k)
            done += 1
            work += n - k  # terms of g_k
        dt = time.perf_counter() - t0
        full = n * (n + 1) / 2
        cpu = {"value": work / full / dt, "unit": "shifts/s", "cores": 1, "kind": "oracle",
               "sample": "%d random output coefficients (%.3g%% of the shift's terms) in %.1f s on one core, "
                         "scaled to one whole shift" % (done, 100 * work / full, dt)}
    line = {"metric": "exact Taylor shifts f(x+1)/s", "value": 1e3 / t_ms, "unit": "shifts/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "taylor: n=16384 coefficients, |f_i| < 2^4096, signed uniform, seed 5",
                       "dispatch": "IPM_COSTMODEL (learned plan per level product)",
                       "output_limbs": ts.limbs, "levels": int(math.log2(n)),
                       "l2": "flushed between timed steps (512 MiB write, outside the events)"},
            "cpu_baseline": cpu, "gpu_launches": int(launches), "launches_per_step": launches / args.steps,
            "clocks": clocks}
    print(json.dumps(line))
    ts.close()
    return 0


FAMILY_GRID = [(d, bits) for d in (64, 256, 1024, 4096) for bits in (32, 256, 2048)]


def run_families(args):
    """Every product family on a grid of balanced shapes (d coefficients
    of `bits` bits, seed d + bits): the chosen form (learned dispatch), the
    analytic planner's 2-D transform, the schoolbook family, Karatsuba over
    y with 1..4 levels, Kronecker substitution and the big-prime form (one
    generalized Fermat prime), each timed on the same
    inputs (CUDA events, L2 flushed) where its limits admit the shape; all
    outputs must agree byte for byte.  The value is the chosen form's
    products/s on the largest shape."""
    import torch
    torch.cuda.set_device(0)
    from paper_1612_05778_gb300 import build as ipm_build
    ipm_build.build()
    import paper_1612_05778_gb300 as ipm
    from paper_1612_05778_gb300 import costmodel as cmod
    cmod.install(points=cmod.load_sweep()["points"])
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    fams = [("chosen", {}, ipm.IPM_COSTMODEL), ("transform", {}, 0), ("school", {"school": 1}, 0)] + \
        [("kara%d" % L, {"kara": L}, 0) for L in (1, 2, 3, 4)] + [("ks", {"ks": 1}, 0), ("bigp", {"bigp": 1}, 0)]
    rows = []
    for d, bits in FAMILY_GRID:
        rng = np.random.default_rng(d + bits)
        a, b = W.random_poly(rng, d, bits), W.random_poly(rng, d, bits)
        da, dan = ipm.to_device(*a)
        db, dbn = ipm.to_device(*b)
        row = {"d": d, "bits": bits, "ms": {}}
        ref = None
        for label, kw, flags in fams:
            try:
                plan = ipm.Plan((d, d, bits, bits), flags=flags, **kw)
            except ipm.IpmError:
                continue  # outside the family's limits
            c, cn = plan.empty_output()
            for _ in range(args.warmup):
                plan.mul(da, dan, db, dbn, c, cn)
            plan.sync()
            row["ms"][label] = timed_ms(torch, lambda: plan.mul(da, dan, db, dbn, c, cn, stream=stream),
                                        args.steps, flush, stream)
            plan.sync()
            if ref is None:
                ref = (c.clone(), cn.clone())
            elif not (torch.equal(ref[0], c) and torch.equal(ref[1], cn)):
                raise SystemExit("family %s disagrees at d=%d bits=%d" % (label, d, bits))
            plan.close()
        others = {k: v for k, v in row["ms"].items() if k != "chosen"}
        row["fastest"] = min(others, key=others.get)
        if "school" in row["ms"]:
            karas = [v for k, v in row["ms"].items() if k.startswith("kara")]
            if karas:
                row["best_karatsuba_over_school"] = row["ms"]["school"] / min(karas)
        rows.append(row)
    top = rows[-1]
    line = {"metric": METRIC, "value": 1e3 / top["ms"]["chosen"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": top["ms"]["chosen"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "families: d in {64, 256, 1024, 4096} x bits in {32, 256, 2048}, balanced, "
                                   "signed uniform, seed d + bits; value = d=4096, 2048-bit"},
            "rows": rows}
    print(json.dumps(line))
    return 0


# The paper's own benchmark (§4, Table classical4andCVL2): random dense
# polynomials with degree d equal to the coefficient size N, CVL_p^2 on a
# 48-core AMD Opteron 6168 (900 MHz), seconds per product.  Context only:
# another machine, another precision of primes.
PAPER_CVL2_SECONDS = {9: 0.152, 10: 0.139, 11: 0.196, 12: 0.295, 13: 0.699, 14: 1.927, 15: 9.138, 16: 33.04}


def run_paper_table(args):
    """The paper's table shapes: d = N = 2^9 .. 2^16 (two polynomials of
    2^k coefficients below 2^(2^k), signed uniform, seed k), each product
    timed through ipm_mul with the plan the learned dispatch picks (the
    planner's where the sweep did not reach); one JSON line whose value is
    the largest shape's products/s, every row with the paper's time beside
    it as context."""
    import torch
    torch.cuda.set_device(0)
    from paper_1612_05778_gb300 import build as ipm_build
    ipm_build.build()
    import paper_1612_05778_gb300 as ipm
    from paper_1612_05778_gb300 import costmodel as cmod
    cmod.install(points=cmod.load_sweep()["points"])
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rows = []
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    l0 = ipm.launch_count()
    for k in sorted(PAPER_CVL2_SECONDS):
        d = 1 << k
        rng = np.random.default_rng(k)
        a = W.random_poly(rng, d, d)
        b = W.random_poly(rng, d, d)
        plan = ipm.Plan((d, d, d, d), flags=ipm.IPM_COSTMODEL)
        da, dan = ipm.to_device(*a)
        db, dbn = ipm.to_device(*b)
        c, cn = plan.empty_output()
        for _ in range(args.warmup):
            plan.mul(da, dan, db, dbn, c, cn)
        plan.sync()
        ms = []
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.mul(da, dan, db, dbn, c, cn, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        plan.sync()
        t = float(np.mean(ms))
        info = plan.info
        rows.append({"d": d, "N": d, "ms": t, "products_per_s": 1e3 / t,
                     "output_gbit_s": info["nc"] * info["lc"] * 32 / (t / 1e3) / 1e9,
                     "plan": {x: info[x] for x in ("K", "M", "r", "Y", "Y2", "S", "Y1b", "kron", "school")},
                     "paper_cvl2_s": PAPER_CVL2_SECONDS[k],
                     "ratio_to_paper": PAPER_CVL2_SECONDS[k] / (t / 1e3)})
        plan.close()
        del da, dan, db, dbn, c, cn
        torch.cuda.empty_cache()
    launches = ipm.launch_count() - l0
    clocks = sampler.stop()
    top = rows[-1]
    line = {"metric": METRIC, "value": top["products_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": top["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "paper_table: d = N = 2^9..2^16 (the paper's Table classical4andCVL2 shapes), "
                                   "signed uniform, seed k; value = d = N = 2^16",
                       "l2": "flushed between timed steps (512 MiB write, outside the events)",
                       "paper_hardware": "48-core AMD Opteron 6168 at 900 MHz, CVL_p^2 (context only)"},
            "rows": rows, "gpu_launches": int(launches), "clocks": clocks}
    print(json.dumps(line))
    return 0


PLAN_KEYS = ("K", "M", "N", "r", "Y", "Y1", "Y2", "S", "Y1b", "kron", "school")


def chosen_flags(ipm, shape, plain_path):
    """The chosen form's plan flags for one product: the learned dispatch
    (committed GB300 cost model and the sweep's table of measured bests),
    or none with plain_path (the analytic planner)."""
    if plain_path:
        return 0, {"source": "planner (--plain)", "params": {}}
    from paper_1612_05778_gb300 import costmodel as cmod
    cmod.install(points=cmod.load_sweep()["points"])
    prm, src = ipm.dispatch(*shape)
    return ipm.IPM_COSTMODEL, {"source": src, "params": prm}


def roofline_of(info, pass_avg, sm_max, traffic_workload=None):
    """Roofline of the dominant pass: its algorithmic integer operations and
    its bytes over its event-timed duration.  The main entry is the bound
    with the larger fraction; beside it the HBM fraction on the method's
    minimal three-pass byte count (in + out + 8R per product, R = r Y K 4)
    and on this implementation's byte count (in + out + 12R), and the same
    two for the whole product."""
    dom = int(np.argmax(pass_avg))
    sbytes, ibytes = schedule_bytes(info), algorithmic_bytes(info)
    aops = algorithmic_int_ops(info)
    peak, peak_kind = load_peak_hbm()
    alu_peak = alu_peak_tops(sm_max)
    secs = pass_avg[dom] / 1e3
    alu_ach = aops[dom] / secs / 1e12
    hbm_s = sbytes[dom] / secs / 1e9
    hbm_i = ibytes[dom] / secs / 1e9
    alu = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "Tops/s (int32)",
           "frac": alu_ach / alu_peak, "peak_kind": "derived: 152 SMs x 128 int32 lanes x %.0f MHz" % sm_max}
    hbm = {"bound": "hbm", "achieved": hbm_s, "peak": peak, "unit": "GB/s", "frac": hbm_s / peak,
           "peak_kind": peak_kind + " (burst copy, MEASURED_PEAKS.json)"}
    main = alu if alu["frac"] >= hbm["frac"] else hbm
    traffic = recorded_traffic(PASS_NAMES[dom], traffic_workload) if traffic_workload else None
    roof = dict(main)
    total_ms = float(np.sum(pass_avg))
    roof.update({
        "kernel": PASS_NAMES[dom], "traffic": traffic,
        "algorithmic_int_ops": aops[dom],
        "hbm": {
            "schedule_bytes": {"bytes": sbytes[dom], "achieved": hbm_s, "peak": peak, "unit": "GB/s",
                               "frac": hbm_s / peak,
                               "what": "the method's three-pass schedule: K1 in + 2R, K2 4R, K3 2R + out"},
            "implementation_bytes": {"bytes": ibytes[dom], "achieved": hbm_i, "peak": peak, "unit": "GB/s",
                                     "frac": hbm_i / peak,
                                     "what": "this implementation: K1 in + 4R, K2 6R, K3 2R + out"},
            "traffic_over_schedule_bytes": (traffic / sbytes[dom]) if traffic else None},
        "product": {"schedule_bytes": sum(sbytes), "implementation_bytes": sum(ibytes), "ms": total_ms,
                    "schedule_frac": sum(sbytes) / (total_ms / 1e3) / 1e9 / peak,
                    "implementation_frac": sum(ibytes) / (total_ms / 1e3) / 1e9 / peak,
                    "alu_frac": sum(aops) / (total_ms / 1e3) / 1e12 / alu_peak},
    })
    return roof


def measure_product(ipm, torch, key, plain_path, steps, warmup, flush, stream, keep=False):
    """One product of workload `key` through ipm_mul with the chosen form's
    plan: event-timed steps (L2 flushed between them), per-pass times, and
    the analytic planner's plan timed beside it when it differs (outputs
    must agree byte for byte)."""
    name, sh, a, b = workload(key)
    shape = (sh.na, sh.nb, sh.bits_a, sh.bits_b)
    flags, dispatch = chosen_flags(ipm, shape, plain_path)
    plan = ipm.Plan(shape, flags=flags)
    info = plan.info
    plain_plan = ipm.Plan(shape)
    same_plan = all(plain_plan.info[k] == info[k] for k in PLAN_KEYS)
    da, dan = ipm.to_device(*a)
    db, dbn = ipm.to_device(*b)
    c, cn = plan.empty_output()
    plan.mul(da, dan, db, dbn, c, cn)
    plan.sync()
    for _ in range(warmup):
        plan.mul(da, dan, db, dbn, c, cn)
    torch.cuda.synchronize()
    plan.set_profiling(True)
    step_ms, pass_ms = [], np.zeros(3)
    l0 = ipm.launch_count()
    for _ in range(steps):
        step_ms.append(timed_ms(torch, lambda: plan.mul(da, dan, db, dbn, c, cn, stream=stream), 1, flush, stream))
        pass_ms += np.array(plan.phase_ms())
    launches = ipm.launch_count() - l0
    plan.set_profiling(False)
    plan.sync()
    plain_ms = None
    if not same_plan:
        c2, cn2 = plain_plan.empty_output()
        for _ in range(warmup):
            plain_plan.mul(da, dan, db, dbn, c2, cn2)
        plain_ms = timed_ms(torch, lambda: plain_plan.mul(da, dan, db, dbn, c2, cn2, stream=stream),
                            max(3, steps // 2), flush, stream)
        plain_plan.sync()
        if not (torch.equal(c, c2) and torch.equal(cn, cn2)):
            raise SystemExit("chosen and plain plans disagree on " + key)
        del c2, cn2
    plain_plan.close()
    ms = float(np.mean(step_ms))
    res = {"name": name, "key": key, "shape": sh, "info": info, "flags": flags, "dispatch": dispatch,
           "step_ms": step_ms, "ms": ms, "value": 1e3 / ms, "pass_avg": pass_ms / steps,
           "plain_ms": plain_ms, "speedup_vs_plain": (plain_ms / ms) if plain_ms else 1.0,
           "launches": launches, "output_gbit_s": sh.nc * sh.lc * 32 / (ms / 1e3) / 1e9}
    if keep:
        res.update({"plan": plan, "a": a, "b": b, "dev": (da, dan, db, dbn), "out": (c, cn)})
    else:
        plan.close()
    return res


def measure_ks_comparator(ipm, torch, steps, flush, stream):
    """The GPU Kronecker-substitution product (ks=1: the integer product
    a(2^s) b(2^s) by the transform path, the paper's KS_s comparator) next
    to the chosen form, on the shapes where KS fits the transform length
    (the small dense workload and the paper's table shapes d = N = 2^9 ..
    2^11); outputs must agree byte for byte."""
    rows = []
    shapes = [("small_dense: d=1024, 255-bit, seed 0", W.small_dense(seed=0))]
    for k in (9, 10, 11):
        rng = np.random.default_rng(k)
        d = 1 << k
        shapes.append(("paper_table: d = N = 2^%d, seed %d" % (k, k),
                       (W.Product(d, d, d, d), W.random_poly(rng, d, d), W.random_poly(rng, d, d))))
    for name, (sh, a, b) in shapes:
        shape = (sh.na, sh.nb, sh.bits_a, sh.bits_b)
        da, dan = ipm.to_device(*a)
        db, dbn = ipm.to_device(*b)
        res = {"workload": name}
        outs = {}
        for label, kw in (("ks", {"ks": 1}), ("chosen", {})):
            flags = 0 if kw else chosen_flags(ipm, shape, False)[0]
            plan = ipm.Plan(shape, flags=flags, **kw)
            c, cn = plan.empty_output()
            for _ in range(3):
                plan.mul(da, dan, db, dbn, c, cn)
            plan.sync()
            res[label + "_ms"] = timed_ms(torch, lambda: plan.mul(da, dan, db, dbn, c, cn, stream=stream),
                                          steps, flush, stream)
            plan.sync()
            outs[label] = (c, cn)
            plan.close()
        if not (torch.equal(outs["ks"][0], outs["chosen"][0]) and torch.equal(outs["ks"][1], outs["chosen"][1])):
            raise SystemExit("Kronecker substitution and the chosen form disagree on " + name)
        res["chosen_over_ks"] = res["ks_ms"] / res["chosen_ms"]
        rows.append(res)
    return {"path": "ks=1: digit polynomials of a(2^s), b(2^s) multiplied by the transform path, slots unpacked",
            "rows": rows}


def product_summary(r, sm_max):
    """The extra-workload entry of the JSON line."""
    info = r["info"]
    return {"workload": r["name"], "value": r["value"], "unit": UNIT, "ms_per_product": r["ms"],
            "output_gbit_s": r["output_gbit_s"], "speedup_vs_plain": r["speedup_vs_plain"],
            "plain_ms": r["plain_ms"],
            "passes_ms": {PASS_NAMES[i]: float(r["pass_avg"][i]) for i in range(3)},
            "plan": {k: info[k] for k in PLAN_KEYS}, "dispatch": r["dispatch"],
            "roofline": roofline_of(info, r["pass_avg"], sm_max, traffic_workload=r["key"])}


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    dist = dist_init(world, "nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1612_05778_gb300 import build as ipm_build
    if rank == 0:
        ipm_build.build()
    barrier(dist)
    import paper_1612_05778_gb300 as ipm

    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(dist)
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    main_r = measure_product(ipm, torch, args.workload, args.plain, args.steps, args.warmup, flush, stream,
                             keep=True)
    torch.cuda.synchronize()
    barrier(dist)
    wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    name, sh, info, plan = main_r["name"], main_r["shape"], main_r["info"], main_r["plan"]
    a, b = main_r["a"], main_r["b"]
    da, dan, db, dbn = main_r["dev"]
    c, cn = main_r["out"]
    flags = main_r["flags"]
    shape = (sh.na, sh.nb, sh.bits_a, sh.bits_b)
    step_ms = main_r["step_ms"]

    # the same plan with every radix-16 stage on the INT8 tensor cores
    # (IPM_TENSOR_STAGES), timed on the same inputs; its output must be
    # byte-identical
    tensor = None
    if not args.no_tensor:
        tplan = ipm.Plan(shape, flags=flags | ipm.IPM_TENSOR_STAGES)
        c3, cn3 = tplan.empty_output()
        for _ in range(max(1, args.warmup // 2)):
            tplan.mul(da, dan, db, dbn, c3, cn3)
        tplan.sync()
        if not (torch.equal(c, c3) and torch.equal(cn, cn3)):
            raise SystemExit("tensor-core stages and integer stages disagree")
        tplan.set_profiling(True)
        tm, tpass = [], np.zeros(3)
        nt = max(3, args.steps // 2)
        for _ in range(nt):
            tm.append(timed_ms(torch, lambda: tplan.mul(da, dan, db, dbn, c3, cn3, stream=stream), 1, flush,
                               stream))
            tpass += np.array(tplan.phase_ms())
        tplan.set_profiling(False)
        tplan.sync()
        tpass /= nt
        tops = tensor_stage_ops(tplan.info, sh.na, sh.nb)
        t_ms = float(np.mean(tm))
        tensor = {"ms_per_step": t_ms, "value": 1e3 / t_ms,
                  "ratio_to_integer_stages": float(np.mean(step_ms)) / t_ms,
                  "passes_ms": {PASS_NAMES[i]: float(tpass[i]) for i in range(3)},
                  "int8_tensor_ops": int(sum(tops)),
                  "int8_tensor": {"achieved": sum(tops) / (t_ms / 1e3) / 1e12, "peak": INT8_MMA_SYNC_TOPS,
                                  "unit": "Tops/s (int8, mma.sync)",
                                  "frac": sum(tops) / (t_ms / 1e3) / 1e12 / INT8_MMA_SYNC_TOPS,
                                  "k_middle_achieved": tops[1] / (tpass[1] / 1e3) / 1e12 if tpass[1] else None,
                                  "peak_kind": "measured mma.sync m16n8k32 u8 microbenchmark"},
                  "path": "IPM_TENSOR_STAGES: radix-16 stages as byte-slice u8 matrix products with "
                          "int32 accumulation (mma.sync), exact Montgomery reduction; output byte-identical"}
        del c3, cn3
        tplan.close()

    local_ms = float(np.sum(step_ms))
    total_ms = max_over_ranks(dist, local_ms, dev)
    ms_per_step = total_ms / args.steps
    value = world * args.steps / (total_ms / 1e3)
    out_bits = sh.nc * sh.lc * 32
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    pass_avg = main_r["pass_avg"]
    roofline = roofline_of(info, pass_avg, sm_max, traffic_workload=args.workload)
    sbytes, abytes, aops = schedule_bytes(info), algorithmic_bytes(info), algorithmic_int_ops(info)
    passes = {PASS_NAMES[i]: {"ms": float(pass_avg[i]), "schedule_bytes": sbytes[i],
                              "implementation_bytes": abytes[i],
                              "gbs_implementation": abytes[i] / (pass_avg[i] / 1e3) / 1e9,
                              "algorithmic_int_ops": aops[i],
                              "int_tops": aops[i] / (pass_avg[i] / 1e3) / 1e12} for i in range(3)}

    # end to end through the host-buffer ABI (pinned host memory): every step
    # copies its inputs in, multiplies and copies its result out, all inside
    # the timed region; E2E_INFLIGHT plans on as many streams keep that many
    # products in flight so their copies overlap the others' compute
    # (ipm_mul_host_async; measured on a GB300: 699 products/s with two,
    # 765 with three, 765 with four on d = 32768, 4096-bit)
    e2e = None
    if not args.no_e2e:
        pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()  # noqa: E731
        ha, han, hb, hbn = pin(a[0]), pin(a[1]), pin(b[0]), pin(b[1])
        nf = E2E_INFLIGHT
        plans = [ipm.Plan(shape, flags=flags) for _ in range(nf)]
        streams = [torch.cuda.Stream() for _ in range(nf)]
        outs = [(torch.empty((info["nc"], info["lc"]), dtype=torch.int32).pin_memory().numpy().view(np.uint32),
                 torch.empty((info["nc"],), dtype=torch.uint8).pin_memory().numpy()) for _ in range(nf)]

        def e2e_steps(k):
            for i in range(k):
                hc, hcn = outs[i % nf]
                plans[i % nf].mul_host_async(ha, han, hb, hbn, hc, hcn, stream=streams[i % nf])
            for pl, st in zip(plans, streams):
                pl.sync(st)

        e2e_steps(2 * nf)
        n_e2e = max(4 * nf, 2 * args.steps)
        barrier(dist)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_steps(n_e2e)
        dt = max_over_ranks(dist, time.perf_counter() - t0, dev)
        if not all(np.array_equal(outs[0][0], o[0]) and np.array_equal(outs[0][1], o[1]) for o in outs[1:]):
            raise SystemExit("end-to-end products disagree")
        if not (np.array_equal(outs[0][0], c.cpu().numpy().view(np.uint32)) and
                np.array_equal(outs[0][1], cn.cpu().numpy())):
            raise SystemExit("end-to-end product differs from the device-resident one")
        h2d = ha.nbytes + han.nbytes + hb.nbytes + hbn.nbytes
        d2h = outs[0][0].nbytes + outs[0][1].nbytes
        e2e = {"value": world * n_e2e / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": n_e2e,
               "api": "ipm_mul_host_async on %d plans and %d streams (pinned host buffers; copies in, "
                      "product, copies out), then ipm_sync; host wall clock" % (nf, nf)}
        for pl in plans:
            pl.close()
        del ha, han, hb, hbn, outs
    del da, dan, db, dbn, c, cn
    plan.close()
    torch.cuda.empty_cache()

    # the other configurations, as extra keys of the same line (rank 0)
    extras = {}
    if rank == 0 and not args.no_extras:
        for key in ("large_dense", "huge_mixed"):
            if key == args.workload:
                continue
            r = measure_product(ipm, torch, key, args.plain, max(5, args.steps // 2), 3, flush, stream)
            extras[key] = product_summary(r, sm_max)
            torch.cuda.empty_cache()
        extras["batch"] = measure_batch(ipm, torch, max(3, args.steps // 4), 3, args.plain, flush)
        torch.cuda.empty_cache()
        extras["ks_comparator"] = measure_ks_comparator(ipm, torch, max(3, args.steps // 4), flush, stream)
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        r = oracle_sample_time(sh, a, b, args.cpu_seconds)
        cpu = {"value": r["products_per_s"], "unit": UNIT, "cores": r["threads"], "kind": "oracle",
               "sample": "%d random output coefficients (%.3g%% of the product's limb products) in "
                         "%.1f s, scaled to one whole product" % (r["coefficients"],
                                                                  100 * r["fraction_of_product"], r["seconds"])}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "output_gbit_s": out_bits * value / 1e9,
        "speedup_vs_plain": main_r["speedup_vs_plain"],
        "plain": ({"ms_per_step": main_r["plain_ms"], "path": "analytic planner's plan"} if main_r["plain_ms"] else
                  {"path": "the analytic planner picks the same plan: one path, ratio 1"}),
        "config": workload_config(name, sh),
        "setup": {"plan": {k: info[k] for k in PLAN_KEYS}, "dispatch": main_r["dispatch"],
                  "primes": info["primes"], "parallelism": "replicas (one product per GPU)",
                  "l2": "flushed between timed steps (512 MiB write, outside the events)",
                  "path": "2-D NTT (Shoup butterflies), %d launches per product" % (
                      3 + (2 if info["Y1b"] > 1 else 0))},
        "roofline": roofline,
        "passes": passes,
        "tensor_stages": tensor,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "extras": extras,
        "batch_speedup_vs_plain": extras["batch"]["speedup_vs_plain"] if "batch" in extras else None,
        "gpu_launches": int(main_r["launches"]),
        "launches_per_step": main_r["launches"] / args.steps,
        "clocks": clocks,
        "wall_s_timed": wall,
    }
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other configurations (d=32768 4096-bit, the mixed d=262144 variant, the batch)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--plain", action="store_true",
                    help="the plain path: analytic planner only, no learned dispatch")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tensor", action="store_true",
                    help="skip timing the tensor-core-stage variant beside the chosen form")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("taylor", "paper_table", "families"):
        # one-GPU measurements: under torchrun only rank 0 runs them
        world, rank, _ = dist_env()
        if world > 1 and rank != 0:
            return 0
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "taylor":
        return run_taylor(args)
    if args.workload == "paper_table":
        return run_paper_table(args)
    if args.workload == "families":
        return run_families(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
