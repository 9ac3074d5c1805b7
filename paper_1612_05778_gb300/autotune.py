"""Exhaustive autotuning sweep over candidate plans.

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


def sweep_point(n: int, bits: int, seed: int, reps: int = 3, max_workspace: float = 120e9,
                check=None) -> dict:
    """Time every candidate plan of the balanced shape (n, n, bits, bits)."""
    import torch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed * 1_000_003 + n * 31 + bits)
    a, an = _operands(torch, n, bits, gen)
    b, bn = _operands(torch, n, bits, gen)
    default = ipm.choose(n, n, bits, bits)
    rec = {"n": n, "bits": bits, "seed": seed, "candidates": []}
    ref = None
    for cand in ipm.candidates(n, n, bits, bits):
        info = cand["info"]
        entry = {"params": cand["params"], "features": cand["features"],
                 "plan": {k: info[k] for k in ("K", "M", "r", "Y", "Y1", "Y2", "S", "Y1b")},
                 "workspace_bytes": info["workspace_bytes"]}
        if info["workspace_bytes"] > max_workspace:
            entry["ms"] = None
            entry["skipped"] = "workspace above %.0f GB" % (max_workspace / 1e9)
            rec["candidates"].append(entry)
            continue
        plan = ipm.Plan((n, n, bits, bits), **cand["params"])
        c, cn = plan.empty_output()
        plan.mul(a, an, b, bn, c, cn)
        torch.cuda.synchronize()
        plan.sync()
        times = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.mul(a, an, b, bn, c, cn)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        entry["ms"] = min(times)
        if ref is None:
            ref = (c, cn)
            if check is not None:
                check(a, an, b, bn, c, cn)
        elif not (torch.equal(ref[0], c) and torch.equal(ref[1], cn)):
            raise AssertionError("candidate %s disagrees with %s at n=%d bits=%d"
                                 % (cand["params"], rec["candidates"][0]["params"], n, bits))
        entry["is_default"] = all(info[k] == default[k] for k in ("K", "M", "r", "Y2", "S", "Y1b"))
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
    ap.add_argument("--check-bits", type=float, default=2**24,
                    help="oracle check (mod 2^61-1 evaluation) when n*bits is at most this")
    args = ap.parse_args(argv)
    import numpy as np
    import oracle

    Q = (1 << 61) - 1
    rng = np.random.default_rng(args.seed)

    def check(a, an, b, bn, c, cn):
        t = int(rng.integers(2, Q - 1))
        h = lambda x, s: (x.cpu().numpy().view(np.uint32), s.cpu().numpy())  # noqa: E731
        A, B, C = h(a, an), h(b, bn), h(c, cn)
        if oracle.eval_mod(C, t, Q) != oracle.eval_mod(A, t, Q) * oracle.eval_mod(B, t, Q) % Q:
            raise AssertionError("product fails c(t) = a(t) b(t) mod 2^61-1")

    grid = W.sweep_grid()
    if args.max_points:
        grid = grid[: args.max_points]
    records = []
    t0 = time.time()

    def fmt(ms):
        return "%.3f ms" % ms if ms is not None else "-"

    for n, bits in grid:
        rec = sweep_point(n, bits, args.seed, args.reps, args.max_workspace,
                          check=check if n * bits <= args.check_bits else None)
        rec["checked_mod_q"] = n * bits <= args.check_bits
        records.append(rec)
        print("n=%7d bits=%5d best %s %s default %s (%d candidates)" % (
            n, bits, fmt(rec["best_ms"]), rec["best_plan"], fmt(rec["default_ms"]),
            len(rec["candidates"])), file=sys.stderr, flush=True)
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
