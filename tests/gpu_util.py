"""Helpers shared by the -m gpu tests: device buffers with a chosen row pitch, and running a tree."""
import numpy as np
import torch

from paper_1510_06585_gb300 import mrw as M


def round_up(v, m):
    return (v + m - 1) // m * m


def to_device(img: np.ndarray, pitch: int | None = None) -> torch.Tensor:
    """Copy a (.., W) uint8 array to the GPU with rows `pitch` bytes apart; returns the (.., W) view."""
    w = img.shape[-1]
    pitch = pitch or round_up(w, 16)
    store = torch.zeros(img.shape[:-1] + (pitch,), dtype=torch.uint8, device="cuda")
    view = store[..., :w]
    view.copy_(torch.from_numpy(np.ascontiguousarray(img)))
    return view


def empty_like_device(img: np.ndarray, pitch: int | None = None, fill: int = 0) -> torch.Tensor:
    w = img.shape[-1]
    pitch = pitch or round_up(w, 16)
    store = torch.full(img.shape[:-1] + (pitch,), fill, dtype=torch.uint8, device="cuda")
    return store[..., :w]


def run_image(tree, img: np.ndarray, cfg=None, pitch=None, reduce_k: int = 0):
    """Execute an image tree on the GPU; returns (output as numpy, reduction or None)."""
    x = to_device(img, pitch)
    y = empty_like_device(img, pitch)
    args = [x, y]
    red = None
    if reduce_k:
        red = torch.full((reduce_k,), -7, dtype=torch.int64, device="cuda")
        args.append(red)
    f = M.execute(tree, args, cfg)
    f.wait(60000)
    out = y.cpu().numpy()
    return out, (red.cpu().numpy() if red is not None else None)


def build_image_tree(names, seeds=None):
    seeds = seeds or {}
    stages = []
    for i, n in enumerate(names):
        stages.append(M.stage(n, seed=seeds.get(i, 0)) if n == "noise" else M.stage(n))
    return M.pipeline(*stages)


def oracle_tree(names, seeds=None):
    seeds = seeds or {}
    return ("pipeline", [("stage", n, {"seed": seeds.get(i, 0)}) for i, n in enumerate(names)])
