"""FP64 oracle of the cost-model MLP — test infrastructure only (see ``oracle/__init__``).

The paper derives configurations for unseen (SCT, workload) pairs from its
knowledge base by scattered-data interpolation (Section 3.2, Configuration
Derivation: an RBF network for 1-3 dimensions, Euclidean nearest neighbour
above). The executor replaces that step by a small learned cost model; the
paper has no counterpart for the network itself, so its definition is the
executor's own:

* 16 -> 64 -> 64 -> K, ReLU after both hidden layers, linear output;
  y[k] = predicted log execution time of configuration k;
* loss = mean over the batch and the K outputs of (y - t)^2, t = measured log time;
* Adam (Kingma and Ba, 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
  w -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps);
* weights are kept in float32 ("master") and rounded to bfloat16
  (round to nearest even) for the forward and backward passes.

Pins (tests/test_oracle_mlp.py): gradients against central finite
differences; the first Adam step against its closed form lr*g/(|g|+eps);
bf16 rounding against exactly representable and tie cases.
"""
from __future__ import annotations

import numpy as np

PARAM_NAMES = ("w1", "b1", "w2", "b2", "w3", "b3")


def init_params(k: int, n_in: int = 16, hidden: int = 64, seed: int = 0) -> dict:
    """He-uniform weights, zero biases, float32."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def he(fan_out, fan_in):
        lim = np.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, size=(fan_out, fan_in)).astype(np.float32)

    return {"w1": he(hidden, n_in), "b1": np.zeros(hidden, np.float32),
            "w2": he(hidden, hidden), "b2": np.zeros(hidden, np.float32),
            "w3": he(k, hidden), "b3": np.zeros(k, np.float32)}


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even); returned as float32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32)


def forward(params: dict, x: np.ndarray):
    """Return (y, cache) in float64 from float64-widened parameters."""
    p = {k: np.asarray(v, dtype=np.float64) for k, v in params.items()}
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ p["w1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["w2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["w3"].T + p["b3"]
    return y, (x, z1, h1, z2, h2)


def loss(params: dict, x: np.ndarray, t: np.ndarray) -> float:
    y, _ = forward(params, x)
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def backward(params: dict, x: np.ndarray, t: np.ndarray) -> dict:
    """Gradients of the mean-squared loss with respect to every parameter (float64)."""
    p = {k: np.asarray(v, dtype=np.float64) for k, v in params.items()}
    y, (xx, z1, h1, z2, h2) = forward(params, x)
    n, k = y.shape
    dy = 2.0 * (y - np.asarray(t, np.float64)) / (n * k)
    g = {"w3": dy.T @ h2, "b3": dy.sum(axis=0)}
    dh2 = dy @ p["w3"]
    dz2 = dh2 * (z2 > 0)
    g["w2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["w2"]
    dz1 = dh1 * (z1 > 0)
    g["w1"] = dz1.T @ xx
    g["b1"] = dz1.sum(axis=0)
    return g


def adam_step(master: dict, grads: dict, m: dict, v: dict, t: int, lr: float,
              b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step (t counts from 1); returns new (master, m, v) in float64."""
    new_w, new_m, new_v = {}, {}, {}
    for k in PARAM_NAMES:
        g = np.asarray(grads[k], np.float64)
        mm = b1 * np.asarray(m[k], np.float64) + (1 - b1) * g
        vv = b2 * np.asarray(v[k], np.float64) + (1 - b2) * g * g
        mhat = mm / (1 - b1 ** t)
        vhat = vv / (1 - b2 ** t)
        new_w[k] = np.asarray(master[k], np.float64) - lr * mhat / (np.sqrt(vhat) + eps)
        new_m[k], new_v[k] = mm, vv
    return new_w, new_m, new_v


def regret(times_chosen: np.ndarray, times_best: np.ndarray) -> np.ndarray:
    """Per-case regret t(chosen) / t(best) - 1."""
    return np.asarray(times_chosen, np.float64) / np.asarray(times_best, np.float64) - 1.0
