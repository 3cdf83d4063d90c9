"""Depth-first skeleton-tree evaluation — test infrastructure only (see ``oracle/__init__``).

Section 2 of the paper: a computation is a skeleton computational tree (SCT)
whose leaves are kernels; on one device the kernels run one after another in a
depth-first walk of the tree (pipeline(K1, loop(K2), K3) runs K1, then K2 as
many times as the loop says, then K3). Pipeline feeds each stage's output to
the next (Section 2.1); Map applies its subtree to independent partitions of
the data (one partition per plane of a volume; the partition's global row
offset is passed on, the Offset trait of Section 3.4); MapReduce adds a
reduction stage whose merging function combines the partial results
(Section 3.4: +, -, x, / or user-defined); Loop repeats its body
(Section 2.1, Loop state: stop condition and carried data).

Trees are plain tuples:
    ("stage", name, params)     name in oracle.image.STAGES or "nbody_accel" / "nbody_kdk"
    ("pipeline", [child, ...])
    ("map", child)
    ("mapreduce", child, op)    op = "add" (the only merging function the executor's
                                device path implements)
    ("loop", child, iters)
    ("loop_while", child, max_iters) repeat while the last run changed its input (at most
                                max_iters runs): a convergence loop on image trees
    ("user", fn)                a user-defined stage (Section 2: the leaves of an SCT are
                                the programmer's kernels): fn(img, y0) returns the stage's
                                output for one plane whose first row has global index y0; the
                                caller writes fn as the plain definition of its kernel

Every intermediate is materialised; ``trace`` records the leaves in the order
they ran. Parity is pinned by tests/test_oracle_skeleton.py (stage order with
non-commuting stages, Map partitions against the whole-volume result).
"""
from __future__ import annotations

import numpy as np

from . import image, nbody


def evaluate_image(tree, img: np.ndarray, trace: list | None = None, y0: int = 0):
    """Evaluate an image-family tree on `img`; returns (output, reduction or None)."""
    kind = tree[0]
    if kind == "stage":
        name, params = tree[1], tree[2] if len(tree) > 2 else {}
        if trace is not None:
            trace.append(name)
        return image.apply_stage(name, img, seed=params.get("seed", 0), y0=y0), None
    if kind == "user":
        if trace is not None:
            trace.append("user")
        if img.ndim == 3:  # a stage sees the rows of a volume as one image, counted across planes
            d, h, w = img.shape
            return np.asarray(tree[1](img.reshape(d * h, w), y0), dtype=np.uint8).reshape(d, h, w), None
        return np.asarray(tree[1](img, y0), dtype=np.uint8), None
    if kind == "pipeline":
        red = None
        for child in tree[1]:
            img, r = evaluate_image(child, img, trace, y0)
            red = r if r is not None else red
        return img, red
    if kind == "map":
        if img.ndim == 3:
            d, h, _ = img.shape
            parts = []
            for k in range(d):
                out, _ = evaluate_image(tree[1], img[k], trace, y0 + k * h)
                parts.append(out)
            return np.stack(parts), None
        return evaluate_image(tree[1], img, trace, y0)
    if kind == "mapreduce":
        out, _ = evaluate_image(("map", tree[1]), img, trace, y0)
        if tree[2] != "add":
            raise ValueError("only the + merging function is defined for the device path")
        if _last_stage(tree[1]) == "threshold3":
            return out, image.class_counts(out, 3)
        return out, image.value_sum(out)
    if kind == "loop":
        red = None
        for _ in range(int(tree[2])):
            img, r = evaluate_image(tree[1], img, trace, y0)
            red = r if r is not None else red
        return img, red
    if kind == "loop_while":
        for _ in range(int(tree[2])):
            out, _ = evaluate_image(tree[1], img, trace, y0)
            changed = not np.array_equal(out, img)
            img = out
            if not changed:
                break
        return img, None
    raise ValueError(f"unknown node {kind!r}")


def _last_stage(tree):
    if tree[0] == "stage":
        return tree[1]
    if tree[0] == "user":
        return "user"
    if tree[0] == "pipeline":
        return _last_stage(tree[1][-1])
    if tree[0] in ("map", "mapreduce", "loop"):
        return _last_stage(tree[1])
    return None


def evaluate_nbody(tree, state, trace: list | None = None):
    """Evaluate an N-body tree on state = (x4 [N,4], v [N,3], a [N,3]) in float64."""
    x4, v, a = state
    kind = tree[0]
    if kind == "stage":
        name, params = tree[1], tree[2]
        if trace is not None:
            trace.append(name)
        g, eps, dt = params["G"], params["eps"], params["dt"]
        if name == "nbody_accel":
            return x4, v, nbody.accel(x4, g, eps)
        if name == "nbody_kdk":
            return nbody.kdk(x4, v, a, 1, g, eps, dt)
        raise ValueError(name)
    if kind == "pipeline":
        for child in tree[1]:
            x4, v, a = evaluate_nbody(child, (x4, v, a), trace)
        return x4, v, a
    if kind == "loop":
        for _ in range(int(tree[2])):
            x4, v, a = evaluate_nbody(tree[1], (x4, v, a), trace)
        return x4, v, a
    raise ValueError(f"node {kind!r} is not part of an N-body tree")
