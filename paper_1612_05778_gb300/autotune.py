"""Exhaustive autotuning sweep over candidate plans.

The points are the balanced grid d = 2^6..2^20 x bits = 2^5..2^14 and 60
seeded unbalanced shapes.

For a product shape, every candidate plan (every valid digit split K with the
planner's tiles and two tile variants, see ``ipm_candidates`` in ipm.h) is
timed with CUDA events on seeded random operands generated on the device.
All candidates must return bit-identical products (every valid plan computes
the same exact c = a*b); a disagreement raises.  The records feed the cost
model (``costmodel.py``) and measure the planner's regret.

    python -m paper_1612_05778_gb300.autotune --out sweep.json [--max-points N]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import paper_1612_05778_gb300 as ipm


def _operands(torch, n: int, bits: int, gen):
    L = (bits + 31) // 32
    limbs = torch.randint(-(2**31), 2**31 - 1, (n, L), dtype=torch.int32, device="cuda", generator=gen)
    rem = bits % 32
    if rem:
        limbs[:, L - 1] &= (1 << rem) - 1
    neg = torch.randint(0, 2, (n,), dtype=torch.uint8, device="cuda", generator=gen)
    neg &= (limbs != 0).any(dim=1).to(torch.uint8)
    return limbs, neg


BATCH = 16                  # batch size of the throughput timings
BATCH_WORKSPACE = 4 << 30   # ... taken when B plans' workspace fits this


def _time(fn, reps):
    import torch
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return min(times)


def sweep_point(shape, seed: int, reps: int = 3, max_workspace: float = 120e9) -> dict:
    """Time every candidate plan of shape (na, nb, bits_a, bits_b): alone
    ("ms") and, where BATCH copies fit BATCH_WORKSPACE, per product in one
    ipm_mul_batched call over BATCH products ("ms_batch")."""
    import torch
    na, nb, ba, bb = shape
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed * 1_000_003 + na * 31 + nb * 7 + ba * 3 + bb)
    a, an = _operands(torch, na, ba, gen)
    b, bn = _operands(torch, nb, bb, gen)
    default = ipm.choose(na, nb, ba, bb)
    rec = {"shape": [na, nb, ba, bb], "n": na, "bits": ba, "seed": seed, "candidates": []}
    ref = None
    for cand in ipm.candidates(na, nb, ba, bb):
        info = cand["info"]
        entry = {"params": cand["params"], "features": cand["features"],
                 "plan": {k: info[k] for k in ("K", "M", "r", "Y", "Y1", "Y2", "S", "Y1b", "kron", "kron_w", "school")},
                 "workspace_bytes": info["workspace_bytes"]}
        if info["workspace_bytes"] > max_workspace:
            entry["ms"] = None
            entry["skipped"] = "workspace above %.0f GB" % (max_workspace / 1e9)
            rec["candidates"].append(entry)
            continue
        plan = ipm.Plan(tuple(shape), **cand["params"])
        c, cn = plan.empty_output()
        plan.mul(a, an, b, bn, c, cn)
        torch.cuda.synchronize()
        plan.sync()
        entry["ms"] = _time(lambda: plan.mul(a, an, b, bn, c, cn), reps)
        if ref is None:
            ref = (c, cn)
        elif not (torch.equal(ref[0], c) and torch.equal(ref[1], cn)):
            raise AssertionError("candidate %s disagrees with %s at %s"
                                 % (cand["params"], rec["candidates"][0]["params"], shape))
        entry["is_default"] = all(info[k] == default[k] for k in ("K", "M", "r", "Y2", "S", "Y1b", "kron", "school"))
        entry["ms_batch"] = None
        if info["workspace_bytes"] * BATCH <= BATCH_WORKSPACE:
            bplan = ipm.Plan([tuple(shape)] * BATCH, **cand["params"])
            outs = [bplan.empty_output(i) for i in range(BATCH)]
            ops = [(a, an, b, bn)] * BATCH
            bplan.mul_batched(ops, outs)
            torch.cuda.synchronize()
            bplan.sync()
            for co, cno in (outs[0], outs[-1]):
                if not (torch.equal(ref[0], co) and torch.equal(ref[1], cno)):
                    raise AssertionError("batched candidate %s disagrees at %s" % (cand["params"], shape))
            entry["ms_batch"] = _time(lambda: bplan.mul_batched(ops, outs), reps) / BATCH
            bplan.close()
            del outs
        rec["candidates"].append(entry)
        plan.close()
        del c, cn
    timed = [c for c in rec["candidates"] if c.get("ms") is not None]
    dflt = [c for c in timed if c.get("is_default")]
    best = min(timed, key=lambda c: c["ms"]) if timed else None
    rec["best_ms"] = best["ms"] if best else None
    rec["best_params"] = best["params"] if best else None
    rec["best_plan"] = best["plan"] if best else None
    rec["default_ms"] = dflt[0]["ms"] if dflt else None
    tb = [c for c in timed if c.get("ms_batch") is not None]
    rec["batch"] = BATCH
    rec["best_ms_batch"] = min(c["ms_batch"] for c in tb) if tb else None
    rec["default_ms_batch"] = dflt[0].get("ms_batch") if dflt else None
    del a, an, b, bn, ref
    torch.cuda.empty_cache()
    return rec


def main(argv=None) -> int:
    import workloads as W

    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--max-points", type=int, default=0)
    ap.add_argument("--max-workspace", type=float, default=120e9,
                    help="skip candidates whose workspace exceeds this many bytes")
    args = ap.parse_args(argv)

    # the balanced grid, then seeded unbalanced shapes
    grid = [(n, n, bits, bits) for n, bits in W.sweep_grid()] + W.sweep_unbalanced(args.seed)
    if args.max_points:
        grid = grid[: args.max_points]
    records = []
    t0 = time.time()

    def fmt(ms):
        return "%.3f ms" % ms if ms is not None else "-"

    for shape in grid:
        rec = sweep_point(shape, args.seed, args.reps, args.max_workspace)
        records.append(rec)
        print("%s best %s %s default %s; batch of %d: best %s default %s (%d candidates)" % (
            shape, fmt(rec["best_ms"]), rec["best_plan"], fmt(rec["default_ms"]), BATCH,
            fmt(rec["best_ms_batch"]), fmt(rec["default_ms_batch"]), len(rec["candidates"])),
            file=sys.stderr, flush=True)
        # rewritten after every point, so an interrupted sweep keeps its data
        with open(args.out + ".tmp", "w") as f:
            json.dump({"device": _device_name(), "seed": args.seed, "seconds": time.time() - t0,
                       "points": records}, f)
        os.replace(args.out + ".tmp", args.out)
    return 0


def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name(0)


if __name__ == "__main__":
    sys.exit(main())
