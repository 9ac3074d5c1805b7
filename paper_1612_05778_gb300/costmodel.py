"""Learned plan dispatch: train the cost model on autotuning sweep records
and judge it by its regret against the exhaustive sweep.

The paper picks its split (DetermineBase, §2.4) by table look-up; here every
candidate plan of a shape (``candidates``: each valid digit split K with the
planner's tiles, plus tile variants) is timed by ``autotune``, and a small
network (``mlp_train``, hand-written CUDA forward/backward/Adam kernels)
learns log2(milliseconds) from the candidates' features.  Dispatch takes
the candidate with the smallest prediction.  Every candidate computes the
same exact product, so the model can cost time but never correctness.

Regret of a choice at a grid point = its measured time / the best measured
time of that point - 1.  Held-out points: every third point of the grid in
sweep order (index % 3 == 2); the model never sees their timings.

    python -m paper_1612_05778_gb300.costmodel --sweep SWEEP.json --out MODEL.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

import paper_1612_05778_gb300 as ipm

DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
SWEEP_GB300 = os.path.join(DATA, "sweep_gb300.json")
MODEL_GB300 = os.path.join(DATA, "costmodel_gb300.json")

_PLAN_KEYS = ("K", "M", "r", "Y2", "S", "Y1b")


def load_sweep(path: str = SWEEP_GB300) -> dict:
    with open(path) as f:
        return json.load(f)


def split_points(points):
    """(training points, held-out points): every third point is held out."""
    train = [p for i, p in enumerate(points) if i % 3 != 2]
    held = [p for i, p in enumerate(points) if i % 3 == 2]
    return train, held


def _timed(point):
    return [c for c in point["candidates"] if c.get("ms") is not None]


def current_features(point):
    """Features of the point's timed candidates as the library computes them
    now (matched by plan), so a model always sees what dispatch will see."""
    now = {tuple(c["info"][k] for k in _PLAN_KEYS): c["features"]
           for c in ipm.candidates(point["n"], point["n"], point["bits"], point["bits"])}
    out = []
    for c in _timed(point):
        key = tuple(c["plan"][k] for k in _PLAN_KEYS)
        out.append(now.get(key, c["features"]))
    return np.asarray(out, dtype=np.float64).reshape(-1, ipm.FEATURES)


def samples(points):
    """Training matrix: one row per timed candidate, target log2(ms)."""
    X, y = [], []
    for p in points:
        feats = current_features(p)
        for f, c in zip(feats, _timed(p)):
            X.append(f)
            y.append(math.log2(c["ms"]))
    return np.asarray(X, dtype=np.float32), np.asarray(y, dtype=np.float32)


def train(points, epochs: int = 4000, lr: float = 1e-3, seed: int = 0):
    """Train on the given points' timings (GPU); returns (model, final mean loss)."""
    X, y = samples(points)
    return ipm.mlp_train(X, y, epochs=epochs, lr=lr, seed=seed)


def choose_by_model(model, point) -> int:
    """Index (among the point's timed candidates) the model would pick."""
    pred = ipm.mlp_predict(model, current_features(point).astype(np.float32))
    return int(np.argmin(pred))


def choose_default(point) -> int:
    """Index of the analytic planner's choice."""
    for i, c in enumerate(_timed(point)):
        if c.get("is_default"):
            return i
    raise KeyError("the planner's choice was not timed at n=%d bits=%d" % (point["n"], point["bits"]))


def regret(point, index: int) -> float:
    t = _timed(point)
    return t[index]["ms"] / min(c["ms"] for c in t) - 1.0


def evaluate(model, points) -> dict:
    """Regret summary of the model and of the analytic planner on `points`."""
    rm = [regret(p, choose_by_model(model, p)) for p in points]
    rd = [regret(p, choose_default(p)) for p in points]

    def summary(r):
        r = np.asarray(r)
        return {"mean": float(r.mean()), "max": float(r.max()), "geomean_slowdown":
                float(np.exp(np.mean(np.log1p(r)))), "optimal_fraction": float(np.mean(r <= 1e-12))}
    return {"points": len(points), "model": summary(rm), "planner": summary(rd),
            "per_point": [{"n": p["n"], "bits": p["bits"], "model": a, "planner": b}
                          for p, a, b in zip(points, rm, rd)]}


def save_model(path: str, model, meta: dict):
    with open(path, "w") as f:
        json.dump({"floats": [float(v) for v in np.asarray(model, dtype=np.float32)], **meta}, f)


def load_model(path: str = MODEL_GB300):
    with open(path) as f:
        d = json.load(f)
    return np.asarray(d["floats"], dtype=np.float32), d


def tuned_entries(points):
    """Tuning-table entries (shape, params of the best measured candidate)."""
    out = []
    for p in points:
        best = min(_timed(p), key=lambda c: c["ms"])
        out.append(((p["n"], p["n"], p["bits"], p["bits"]), best["params"]))
    return out


def install(model=None, points=None):
    """Install a model (default: the committed GB300 model) and, when sweep
    points are given, the tuning table of their measured bests."""
    if model is None:
        model, _ = load_model()
    ipm.set_cost_model(model)
    if points is not None:
        ipm.set_tuned(tuned_entries(points))


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--sweep", default=SWEEP_GB300)
    ap.add_argument("--out", default=None, help="write the trained model (JSON)")
    ap.add_argument("--epochs", type=int, default=4000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)
    sweep = load_sweep(args.sweep)
    tr, held = split_points(sweep["points"])
    model, loss = train(tr, args.epochs, args.lr, args.seed)
    ev = evaluate(model, held)
    ev_train = evaluate(model, tr)
    print(json.dumps({"train_points": len(tr), "held_out_points": len(held), "final_loss": loss,
                      "held_out": {k: ev[k] for k in ("model", "planner")},
                      "train": {k: ev_train[k] for k in ("model", "planner")}}, indent=1))
    if args.out:
        save_model(args.out, model, {"device": sweep.get("device"), "epochs": args.epochs, "lr": args.lr,
                                     "seed": args.seed, "final_loss": loss, "sweep": os.path.basename(args.sweep),
                                     "held_out": {k: ev[k] for k in ("model", "planner")}})
    return 0


if __name__ == "__main__":
    sys.exit(main())
