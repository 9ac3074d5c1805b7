"""Host-side tests of the learned plan dispatch (no GPU).

* The CPU reference network (oracle/mlp.py) is pinned to calculus: its
  gradient must match central finite differences of its loss, and a network
  whose output weights are zero must predict the closed form y_mean + b3*y_sd.
* ipm_candidates: every candidate plans to what it claims, the analytic
  planner's choice is among them, candidates are distinct, features finite.
* The regret bookkeeping of costmodel.py on a hand-made sweep record.
"""
import math

import numpy as np
import pytest

import paper_1612_05778_gb300 as ipm
from oracle import mlp as omlp
from paper_1612_05778_gb300 import costmodel as cm


def _data(rng, n=40):
    X = rng.normal(size=(n, omlp.F)) * rng.uniform(0.5, 3, omlp.F) + rng.uniform(-2, 2, omlp.F)
    y = X[:, 0] - 0.5 * X[:, 3] + np.sin(X[:, 5]) + 0.1 * rng.normal(size=n)
    return X, y


def test_layout_matches_library_constants():
    assert omlp.NPARAM == ipm.MLP_PARAMS
    assert omlp.NFLOATS == ipm.MLP_FLOATS
    assert omlp.F == ipm.FEATURES and omlp.H == ipm.MLP_HIDDEN


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_reference_gradient_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    X, y = _data(rng)
    model = omlp.random_model(rng, X, y)
    L, g = omlp.grad(model, X, y)
    assert L == pytest.approx(omlp.loss(model, X, y), rel=1e-12)
    h = 1e-6
    base = 2 * omlp.F + 2
    # every parameter of the output layers, a strided sample of the rest
    idx = list(range(0, omlp.NPARAM, 7)) + list(range(omlp.NPARAM - 2 * omlp.H - 1, omlp.NPARAM))
    for i in idx:
        mp = model.copy()
        mm = model.copy()
        mp[base + i] += h
        mm[base + i] -= h
        fd = (omlp.loss(mp, X, y) - omlp.loss(mm, X, y)) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-6), i


def test_reference_zero_output_layer_predicts_bias():
    rng = np.random.default_rng(5)
    X, y = _data(rng)
    model = omlp.random_model(rng, X, y)
    _, _, y_mean, y_sd, _ = omlp.unpack(model)
    model[2 * omlp.F + 2 + omlp.NPARAM - omlp.H - 1: -1] = 0.0   # w3 = 0
    model[-1] = 0.75                                              # b3
    np.testing.assert_allclose(omlp.predict(model, X), y_mean + 0.75 * y_sd, rtol=1e-12)
    # then only b3 has a gradient, equal to sum(o - t)
    L, g = omlp.grad(model, X, y)
    t = (y - y_mean) / y_sd
    assert g[-1] == pytest.approx(np.sum(0.75 - t), rel=1e-12)
    assert np.all(g[:-1 - omlp.H] == 0)


def test_reference_linear_regime():
    """With every pre-activation positive the network is affine in z, so the
    W1 gradient is d1^T z computed by hand."""
    rng = np.random.default_rng(9)
    X, y = _data(rng, 8)
    model = omlp.random_model(rng, X, y)
    base = 2 * omlp.F + 2
    F, H = omlp.F, omlp.H
    model[base:base + H * F] = 0.0                       # W1 = 0
    model[base + H * F:base + H * F + H] = 1.0           # b1 = 1 -> h1 = 1
    W2 = model[base + H * F + H:base + H * F + H + H * H].reshape(H, H)
    W2[:] = np.abs(W2)                                   # keep layer 2 active
    _, g = omlp.grad(model, X, y)
    _, inv_sd, y_mean, y_sd, P = omlp.unpack(model)
    z = (X - model[:F]) * inv_sd
    o = np.full(len(X), P["w3"] @ np.maximum(P["W2"] @ np.ones(H) + P["b2"], 0) + P["b3"])
    d = o - (y - y_mean) / y_sd
    d1 = np.outer(d, P["w3"] @ P["W2"])                  # dL/d(layer-1 pre-activation)
    np.testing.assert_allclose(g[:H * F].reshape(H, F), d1.T @ z, rtol=1e-10, atol=1e-12)


SHAPES = [(64, 64, 32, 32), (1024, 1024, 256, 256), (4096, 4096, 4096, 4096), (65536, 65536, 64, 64),
          (300, 2000, 17, 900), (1 << 20, 1 << 20, 32, 32)]


@pytest.mark.parametrize("shape", SHAPES)
def test_candidates_are_valid_distinct_and_include_the_planner(shape):
    cands = ipm.candidates(*shape)
    assert len(cands) >= 1
    keys = set()
    for c in cands:
        info = ipm.choose(*shape, **c["params"])
        assert info == c["info"]
        key = tuple(info[k] for k in ("K", "M", "r", "Y2", "S", "Y1b", "kron", "school"))
        assert key not in keys
        keys.add(key)
        assert len(c["features"]) == ipm.FEATURES
        assert all(math.isfinite(v) for v in c["features"])
        assert c["features"][4] == pytest.approx(math.log2(max(info["K"], 1)))
        assert c["features"][6] == info["r"]
    d = ipm.choose(*shape)
    assert tuple(d[k] for k in ("K", "M", "r", "Y2", "S", "Y1b", "kron", "school")) in keys


def test_candidates_reject_bad_shape():
    lib = ipm.load_library()
    assert lib.ipm_candidates(None, None, 0) < 0
    bad = ipm.Shape(-1, 3, 32, 32)
    assert lib.ipm_candidates(bad, None, 0) == -1


def _fake_point(n, bits, times, default):
    cands = []
    for i, t in enumerate(times):
        cands.append({"params": {"K": 2 << i}, "plan": {"K": 2 << i}, "features": [0.0] * 16,
                      "ms": t, "is_default": i == default})
    cands.append({"params": {"K": 1 << 12}, "ms": None, "skipped": "workspace"})
    return {"n": n, "bits": bits, "candidates": cands}


def test_regret_bookkeeping():
    p = _fake_point(64, 32, [2.0, 1.0, 4.0], default=0)
    assert cm.choose_default(p) == 0
    assert cm.regret(p, 0) == pytest.approx(1.0)
    assert cm.regret(p, 1) == 0.0
    assert cm.regret(p, 2) == pytest.approx(3.0)
    pts = [_fake_point(64 << i, 32, [1.0, 2.0], 0) for i in range(7)]
    tr, held = cm.split_points(pts)
    assert [p["n"] for p in held] == [64 << 2, 64 << 5]
    assert len(tr) == 5
    ent = cm.tuned_entries([p])
    assert ent == [((64, 64, 32, 32), {"K": 4})]
