"""Learned plan dispatch: train the cost model on autotuning sweep records
and measure it by its regret against the exhaustive sweep.

The paper picks its split (DetermineBase, §2.4) by table look-up; here every
candidate plan of a shape (``candidates``: each valid digit split K with the
planner's tiles, plus tile variants) is timed by ``autotune``, and a small
network (``mlp_train``, hand-written CUDA forward/backward/Adam kernels)
learns log2(milliseconds per product) from the candidates' features, for
products run alone and inside a batch (the last feature is log2 of the
batch size, capped at 16).  Dispatch takes the candidate with the smallest
prediction.  Every candidate computes the
same exact product, so the model can cost time but never correctness.

Regret of a choice at a sweep point = its measured time / the best measured
time of that point - 1.  Held-out points: every third point in sweep order
(index % 3 == 2), of the balanced grid and of the unbalanced shapes alike;
the model never sees their timings.

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

_PLAN_KEYS = ("K", "M", "r", "Y2", "S", "Y1b", "kron", "school")
_PLAN_DEFAULTS = {"kron": 1, "school": 0}  # for records written before these keys existed


def load_sweep(path: str = SWEEP_GB300) -> dict:
    with open(path) as f:
        return json.load(f)


def split_points(points):
    """(training points, held-out points): every third point is held out."""
    train = [p for i, p in enumerate(points) if i % 3 != 2]
    held = [p for i, p in enumerate(points) if i % 3 == 2]
    return train, held


def _key(batch: int) -> str:
    return "ms" if batch == 1 else "ms_batch"


def _timed(point, batch: int = 1):
    k = _key(batch)
    return [c for c in point["candidates"] if c.get(k) is not None]


def batch_feature(batch: int) -> float:
    """Value of the batch-size feature (log2 of the batch size, capped at 16)."""
    return math.log2(min(batch, 16))


def shape_of(point):
    """(na, nb, bits_a, bits_b) of a sweep record."""
    if "shape" in point:
        return tuple(point["shape"])
    return (point["n"], point["n"], point["bits"], point["bits"])


def current_features(point, batch: int = 1):
    """Features of the point's candidates timed at this batch size, as the
    library computes them now (matched by plan), so a model always sees what
    dispatch will see."""
    now = {tuple(c["info"][k] for k in _PLAN_KEYS): c["features"]
           for c in ipm.candidates(*shape_of(point))}
    out = []
    for c in _timed(point, batch):
        key = tuple(c["plan"].get(k, _PLAN_DEFAULTS.get(k)) for k in _PLAN_KEYS)
        f = list(now.get(key, c["features"]))[:ipm.FEATURES]
        f += [0.0] * (ipm.FEATURES - len(f))
        f[ipm.FEATURES - 1] = batch_feature(batch)
        out.append(f)
    return np.asarray(out, dtype=np.float64).reshape(-1, ipm.FEATURES)


def batch_sizes(points):
    """The batch sizes timed in a sweep: 1 and the sweep's batch, if any."""
    b = {p.get("batch", 1) for p in points if any(c.get("ms_batch") is not None for c in p["candidates"])}
    return [1] + sorted(x for x in b if x > 1)


def samples(points):
    """Training matrix: one row per timed (candidate, batch size), target
    log2(milliseconds per product)."""
    X, y = [], []
    for batch in batch_sizes(points):
        for p in points:
            if batch > 1 and p.get("batch") != batch:
                continue
            feats = current_features(p, batch)
            for f, c in zip(feats, _timed(p, batch)):
                X.append(f)
                y.append(math.log2(c[_key(batch)]))
    return np.asarray(X, dtype=np.float32), np.asarray(y, dtype=np.float32)


def train(points, epochs: int = 8000, lr: float = 1e-3, seed: int = 0):
    """Train on the given points' timings (GPU); returns (model, final mean loss)."""
    X, y = samples(points)
    return ipm.mlp_train(X, y, epochs=epochs, lr=lr, seed=seed)


def choose_by_model(model, point, batch: int = 1) -> int:
    """Index (among the point's candidates timed at this batch size) the
    model would pick."""
    pred = ipm.mlp_predict(model, current_features(point, batch).astype(np.float32))
    return int(np.argmin(pred))


def choose_default(point, batch: int = 1) -> int:
    """Index of the analytic planner's choice."""
    for i, c in enumerate(_timed(point, batch)):
        if c.get("is_default"):
            return i
    raise KeyError("the planner's choice was not timed at %s" % (shape_of(point),))


def regret(point, index: int, batch: int = 1) -> float:
    t = _timed(point, batch)
    k = _key(batch)
    return t[index][k] / min(c[k] for c in t) - 1.0


def _summary(r):
    r = np.asarray(r)
    return {"mean": float(r.mean()), "max": float(r.max()), "geomean_slowdown":
            float(np.exp(np.mean(np.log1p(r)))), "optimal_fraction": float(np.mean(r <= 1e-12))}


def evaluate(model, points, batch: int = 1) -> dict:
    """Regret summary of the model and of the analytic planner on the
    points timed at this batch size."""
    pts = [p for p in points if _timed(p, batch) and any(c.get("is_default") for c in _timed(p, batch))]
    rm = [regret(p, choose_by_model(model, p, batch), batch) for p in pts]
    rd = [regret(p, choose_default(p, batch), batch) for p in pts]
    return {"batch": batch, "points": len(pts), "model": _summary(rm), "planner": _summary(rd),
            "per_point": [{"shape": shape_of(p), "model": a, "planner": b} for p, a, b in zip(pts, rm, rd)]}


def save_model(path: str, model, meta: dict):
    with open(path, "w") as f:
        json.dump({"floats": [float(v) for v in np.asarray(model, dtype=np.float32)], **meta}, f)


def load_model(path: str = MODEL_GB300):
    with open(path) as f:
        d = json.load(f)
    return np.asarray(d["floats"], dtype=np.float32), d


def tuned_entries(points):
    """Tuning-table entries (shape, params of the best measured candidate
    that still plans with this library: the tile limits may have changed
    since the sweep)."""
    out = []
    for p in points:
        for c in sorted(_timed(p), key=lambda c: c["ms"]):
            try:
                ipm.choose(*shape_of(p), **c["params"])
            except ipm.IpmError:
                continue
            out.append((shape_of(p), c["params"]))
            break
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
    ap.add_argument("--epochs", type=int, default=8000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)
    sweep = load_sweep(args.sweep)
    tr, held = split_points(sweep["points"])
    model, loss = train(tr, args.epochs, args.lr, args.seed)
    keep = ("batch", "points", "model", "planner")
    report = {"train_points": len(tr), "held_out_points": len(held), "final_loss": loss,
              "held_out": [{k: evaluate(model, held, b)[k] for k in keep} for b in batch_sizes(held)],
              "train": [{k: evaluate(model, tr, b)[k] for k in keep} for b in batch_sizes(tr)]}
    print(json.dumps(report, indent=1))
    if args.out:
        save_model(args.out, model, {"device": sweep.get("device"), "epochs": args.epochs, "lr": args.lr,
                                     "seed": args.seed, "final_loss": loss, "sweep": os.path.basename(args.sweep),
                                     "held_out": report["held_out"]})
    return 0


if __name__ == "__main__":
    sys.exit(main())
