"""Learned configuration derivation: data collection, training and regret evaluation.

The paper derives a configuration for an unseen (SCT, workload) pair from its knowledge base by
scattered-data interpolation: an RBF network for 1-3 dimensions, Euclidean nearest neighbour above
(Section 3.2, Configuration Derivation), and builds profiles by a timed search (Algorithm 1). Here:

* the exhaustive autotuner (``mrw_tune_measure``) times all 16 candidate configurations of random
  compound skeletons (1-6 stages, 2^12..2^28 elements, u8 image stages or f32 saxpy) on the GPU;
* the cost model (``mrw_model_*``: MLP 16 -> 64 -> 64 -> 16, bf16 weights, fp32 accumulation,
  hand-written forward / backward / Adam kernels) is trained on those measurements to predict each
  configuration's log time relative to the sample's mean log time;
* on held-out skeletons its choice (argmin of the predicted times) is scored by regret
  t(chosen) / t(best) - 1 against the exhaustive best, beside the default configuration and the
  paper's nearest-neighbour derivation over the training set.

Everything that computes runs in libmrw's kernels; this module only generates the workloads,
standardises features (host-side input preparation) and keeps the bookkeeping.

Usage: python -m paper_1510_06585_gb300.costmodel --train 20000 --test 1000 --out results.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs
from . import mrw as M

MAX_IMAGE_ELEMS = 1 << 28
MAX_SAXPY_ELEMS = 1 << 26


class Arena:
    """Device buffers reused by every sample (the largest workload's size)."""

    def __init__(self, max_log2: int):
        import torch
        self.torch = torch
        n = min(1 << max_log2, MAX_IMAGE_ELEMS)
        # rows are padded to 16 bytes: a pitch is at most 1.25x the width for the widths drawn (>= 64)
        self.img_in = torch.randint(0, 256, (n + (n >> 2) + 4096,), dtype=torch.uint8, device="cuda")
        self.img_out = torch.empty_like(self.img_in)
        ns = min(1 << max_log2, MAX_SAXPY_ELEMS)
        self.x = torch.rand(ns, device="cuda")
        self.y = torch.rand(ns, device="cuda")
        self.counts = torch.zeros(3, dtype=torch.int64, device="cuda")

    def image_views(self, rows: int, width: int):
        pitch = (width + 15) // 16 * 16
        need = rows * pitch
        if need > self.img_in.numel():
            raise ValueError("sample larger than the arena")
        a = self.img_in[:need].view(rows, pitch)[:, :width]
        b = self.img_out[:need].view(rows, pitch)[:, :width]
        return a, b


def build_tree(spec):
    """mrw tree for one random skeleton description (see inputs.random_skeletons)."""
    if spec["kind"] == "saxpy":
        return M.map_(M.stage("saxpy", alpha=1.5))
    stages = []
    for i, name in enumerate(spec["stages"]):
        if name == "noise":
            stages.append(M.stage("noise", seed=spec["seed"] + i))
        else:
            stages.append(M.stage(name))
    body = M.pipeline(*stages)
    if spec["kind"] == "map":
        return M.map_(body)
    if spec["kind"] == "mapreduce":
        return M.mapreduce(M.map_(body))
    return body


def sample_args(arena: Arena, spec):
    if spec["kind"] == "saxpy":
        n = min(spec["width"] * spec["rows"], MAX_SAXPY_ELEMS)
        return [arena.x[:n], arena.y[:n]]
    a, b = arena.image_views(spec["rows"], spec["width"])
    args = [a, b]
    if spec["kind"] == "mapreduce":
        args.append(arena.counts)
    return args


def collect(n: int, seed: int, max_log2: int = 28, reps: int = 3, arena: Arena | None = None, log=None):
    """Features [n, 16] and measured times [n, 16] (ms) of n random skeletons (all 16 configs)."""
    specs = inputs.random_skeletons(n, seed=seed, max_log2=max_log2)
    arena = arena or Arena(max_log2)
    feats = np.zeros((n, M.MRW_NFEATURES), np.float32)
    times = np.zeros((n, 16), np.float64)
    t0 = time.time()
    for i, spec in enumerate(specs):
        tree = build_tree(spec)
        args = sample_args(arena, spec)
        feats[i] = M.features(tree, args)
        cfgs = M.tune_candidates(tree, args)
        t = M.tune_measure(tree, args, cfgs, reps=reps)
        bad = t <= 0
        if bad.all():
            raise RuntimeError(f"no valid configuration for sample {i}: {spec}")
        t[bad] = t[~bad].max() * 10.0
        times[i] = t
        if log and (i + 1) % 1000 == 0:
            log(f"collected {i + 1}/{n} in {time.time() - t0:.1f}s")
    return feats, times, specs


def targets(times: np.ndarray) -> np.ndarray:
    """Per-sample centred log times: the model only has to rank the configurations."""
    lt = np.log(times)
    return (lt - lt.mean(axis=1, keepdims=True)).astype(np.float32)


class Standardizer:
    def __init__(self, x: np.ndarray):
        self.mu = x.mean(axis=0)
        self.sd = x.std(axis=0)
        self.sd[self.sd < 1e-6] = 1.0

    def __call__(self, x: np.ndarray) -> np.ndarray:
        return ((x - self.mu) / self.sd).astype(np.float32)


def train(feats, times, epochs=300, batch=256, lr=2e-3, hidden=64, seed=0):
    import torch
    std = Standardizer(feats)
    model = M.Model(16, hidden, seed=seed)
    xd = torch.from_numpy(std(feats)).cuda()
    td = torch.from_numpy(targets(times)).cuda()
    t0 = time.time()
    loss = model.train(xd, td, epochs=epochs, batch=batch, lr=lr, seed=seed)
    torch.cuda.synchronize()
    return model, std, loss, time.time() - t0


def predict(model, std, feats) -> np.ndarray:
    import torch
    xd = torch.from_numpy(std(feats)).cuda()
    y = torch.zeros(feats.shape[0], 16, device="cuda")
    model.forward(xd, y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def fold_standardization(model, std) -> None:
    """Fold the feature standardisation into the first layer so the model takes raw features
    (what mrw_features returns), e.g. before installing it with mrw_tune_set_model:
    W1 (x - mu) / sd + b1 = (W1 / sd) x + (b1 - (W1 / sd) mu)."""
    p = M.unpack_params(model.get_params(), model.k, model.hidden)
    w1 = p["w1"].astype(np.float64) / std.sd[None, :]
    p["b1"] = (p["b1"] - w1 @ std.mu).astype(np.float32)
    p["w1"] = w1.astype(np.float32)
    model.set_params(M.pack_params(p))


def regret_of(choice: np.ndarray, times: np.ndarray) -> np.ndarray:
    best = times.min(axis=1)
    return times[np.arange(len(choice)), choice] / best - 1.0


def nearest_neighbour_choice(train_feats, train_times, std, test_feats) -> np.ndarray:
    """The paper's derivation for more than 3 dimensions: the best configuration of the training
    sample nearest in (standardised) feature space."""
    a = std(train_feats)
    b = std(test_feats)
    best = train_times.argmin(axis=1)
    out = np.zeros(len(b), np.int64)
    for i in range(0, len(b), 256):
        d = ((b[i:i + 256, None, :] - a[None, :, :]) ** 2).sum(axis=2)
        out[i:i + 256] = best[d.argmin(axis=1)]
    return out


def summary(r: np.ndarray) -> dict:
    return {"mean": float(r.mean()), "median": float(np.median(r)), "p90": float(np.percentile(r, 90)),
            "within_10pct": float((r <= 0.10).mean())}


def experiment(n_train: int, n_test: int, max_log2: int = 28, epochs: int = 300, reps: int = 3, log=print):
    arena = Arena(max_log2)
    t0 = time.time()
    ftr, ttr, _ = collect(n_train, inputs.SEED_MODEL, max_log2, reps, arena, log)
    fte, tte, _ = collect(n_test, inputs.SEED_MODEL + 1000, max_log2, reps, arena, log)
    t_collect = time.time() - t0
    model, std, loss, t_train = train(ftr, ttr, epochs=epochs)
    pred = predict(model, std, fte)
    choice = pred.argmin(axis=1)
    res = {
        "n_train": n_train, "n_test": n_test, "max_log2": max_log2, "epochs": epochs, "reps": reps,
        "collect_seconds": round(t_collect, 1), "train_seconds": round(t_train, 2), "final_train_loss": loss,
        "learned": summary(regret_of(choice, tte)),
        "default_config": summary(regret_of(np.zeros(n_test, np.int64), tte)),
        "nearest_neighbour_kb": summary(regret_of(nearest_neighbour_choice(ftr, ttr, std, fte), tte)),
        "random_config": summary(regret_of(np.random.Generator(np.random.PCG64(0)).integers(0, 16, n_test), tte)),
        "oracle_best_is_fused": float((tte.argmin(axis=1) < 8).mean()),
    }
    return res, model, std


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--test", type=int, default=1000)
    ap.add_argument("--max-log2", type=int, default=28)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res, _, _ = experiment(a.train, a.test, a.max_log2, a.epochs, a.reps)
    txt = json.dumps(res, indent=1)
    print(txt)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt + "\n")


if __name__ == "__main__":
    main()
