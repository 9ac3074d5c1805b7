"""CPU reference of the plan cost model -- TEST INFRASTRUCTURE ONLY.

Only tests/ may import this module.  It restates, in float64 numpy, the
network the CUDA library trains and evaluates for its learned plan dispatch
(the paper has no such model; its DetermineBase, §2.4, uses a table), so the
GPU's forward pass and gradient can be checked against it.  It shares no code
with the library.

Network on standardised inputs z = (x - mean) * inv_sd:
    h1 = relu(W1 z + b1), h2 = relu(W2 h1 + b2), o = w3 . h2 + b3,
loss over samples = sum 1/2 (o - t)^2 with t = (y - y_mean) / y_sd, and the
prediction in target units o * y_sd + y_mean.

Model vector (float32 in the library): means [F], inverse sds [F], y_mean,
y_sd, then W1 [H][F], b1 [H], W2 [H][H], b2 [H], w3 [H], b3.
"""
from __future__ import annotations

import numpy as np

F = 19
H = 32
NPARAM = H * F + H + H * H + H + H + 1
NFLOATS = 2 * F + 2 + NPARAM


def unpack(model):
    """Split a model vector into its named parts (float64 copies)."""
    m = np.asarray(model, dtype=np.float64)
    assert m.shape == (NFLOATS,)
    mean, inv_sd = m[:F], m[F:2 * F]
    y_mean, y_sd = m[2 * F], m[2 * F + 1]
    p = m[2 * F + 2:]
    o = 0
    parts = {}
    for name, shape in (("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", ())):
        size = int(np.prod(shape)) if shape else 1
        parts[name] = p[o:o + size].reshape(shape) if shape else p[o]
        o += size
    return mean, inv_sd, y_mean, y_sd, parts


def forward(model, X):
    """Standardised outputs o[n] and the activations (z, h1, h2)."""
    mean, inv_sd, _, _, P = unpack(model)
    z = (np.asarray(X, dtype=np.float64) - mean) * inv_sd
    h1 = np.maximum(z @ P["W1"].T + P["b1"], 0.0)
    h2 = np.maximum(h1 @ P["W2"].T + P["b2"], 0.0)
    return h2 @ P["w3"] + P["b3"], (z, h1, h2)


def predict(model, X):
    """Predictions in target units."""
    _, _, y_mean, y_sd, _ = unpack(model)
    return forward(model, X)[0] * y_sd + y_mean


def loss(model, X, y):
    """Sum over samples of 1/2 (o - t)^2."""
    _, _, y_mean, y_sd, _ = unpack(model)
    o, _ = forward(model, X)
    t = (np.asarray(y, dtype=np.float64) - y_mean) / y_sd
    return 0.5 * float(np.sum((o - t) ** 2))


def grad(model, X, y):
    """(loss, gradient over the NPARAM parameters) by the chain rule."""
    _, _, y_mean, y_sd, P = unpack(model)
    o, (z, h1, h2) = forward(model, X)
    t = (np.asarray(y, dtype=np.float64) - y_mean) / y_sd
    d = o - t                                   # dL/do per sample
    g_b3 = d.sum()
    g_w3 = d @ h2
    d2 = np.outer(d, P["w3"]) * (h2 > 0)        # dL/d(W2 h1 + b2)
    g_W2 = d2.T @ h1
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ P["W2"]) * (h1 > 0)              # dL/d(W1 z + b1)
    g_W1 = d1.T @ z
    g_b1 = d1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return 0.5 * float(np.sum(d * d)), g


def random_model(rng, X=None, y=None, scale=0.5):
    """A model with random parameters; standardisation from (X, y) if given."""
    m = np.zeros(NFLOATS)
    if X is not None:
        X = np.asarray(X, dtype=np.float64)
        m[:F] = X.mean(axis=0)
        sd = X.std(axis=0)
        m[F:2 * F] = np.where(sd > 1e-6, 1.0 / np.maximum(sd, 1e-6), 0.0)
    else:
        m[F:2 * F] = 1.0
    if y is not None:
        m[2 * F] = float(np.mean(y))
        m[2 * F + 1] = max(float(np.std(y)), 1e-6)
    else:
        m[2 * F + 1] = 1.0
    m[2 * F + 2:] = rng.uniform(-scale, scale, NPARAM)
    return m
