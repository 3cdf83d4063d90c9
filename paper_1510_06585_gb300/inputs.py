"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module only draws numbers; it holds none of the skeleton stages' arithmetic.
Every generator is numpy's PCG64 (O'Neill 2014), whose output is identical on
x86 and Arm, so the same seed gives the same bytes on every machine.

Workload shapes follow the benchmarks of Section 4 of the paper (Filter
Pipeline on greyscale images, Segmentation of a 3-D greyscale volume, direct-sum
N-body) at the sizes this executor is measured on:

* filter image   : H x W uint8, uniform in [0, 255]                       (seed 1)
* segmentation   : D x H x W uint8, 3-component normal mixture, means
                   40/128/220, sd 15, equal weights, rounded half-to-even and
                   clamped to [0, 255]; drawn in chunks of 16 planes, chunk c
                   from PCG64([seed, c]) so any sub-volume is reproducible   (seed 3)
* n-body         : positions uniform in the unit cube, masses uniform in
                   [0.5, 1], drawn in float64 and rounded to float32; the
                   state is three float32 [N, 4] arrays x=(x,y,z,m),
                   v=(vx,vy,vz,0), a=(ax,ay,az,0), v = 0                     (seed 4)
* batch          : n images with sides W, H independently log-uniform in
                   [64, 2048] (rounded), rows padded to a 16-byte pitch,
                   each instance 256-byte aligned in one arena; instance i's
                   pixels from PCG64(5_000_000 + i), its noise seed 2 + i    (seed 5)
* random skeletons for the cost model                                        (seed 6)
* fft signals    : nfft x N complex64, real and imaginary parts uniform in
                   [-1, 1), drawn in float64 and rounded to float32          (seed 7)
"""
from __future__ import annotations

import math

import numpy as np

SEED_IMAGE = 1
SEED_NOISE = 2
SEED_VOLUME = 3
SEED_NBODY = 4
SEED_BATCH = 5
SEED_MODEL = 6
SEED_FFT = 7

VOLUME_MEANS = (40.0, 128.0, 220.0)
VOLUME_SD = 15.0
VOLUME_CHUNK = 16  # planes per independently seeded chunk


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def filter_image(h: int, w: int, seed: int = SEED_IMAGE) -> np.ndarray:
    """Uniform uint8 greyscale image of shape (h, w)."""
    return _rng(seed).integers(0, 256, size=(h, w), dtype=np.uint8)


def volume(d: int, h: int, w: int, seed: int = SEED_VOLUME, out: np.ndarray | None = None) -> np.ndarray:
    """3-component mixture volume (d, h, w) uint8; plane chunks are seeded independently."""
    if out is None:
        out = np.empty((d, h, w), dtype=np.uint8)
    means = np.asarray(VOLUME_MEANS)
    for c0 in range(0, d, VOLUME_CHUNK):
        c1 = min(d, c0 + VOLUME_CHUNK)
        rng = _rng([seed, c0 // VOLUME_CHUNK])
        shape = (c1 - c0, h, w)
        comp = rng.integers(0, 3, size=shape, dtype=np.int8)
        vals = rng.normal(0.0, 1.0, size=shape)
        vals *= VOLUME_SD
        vals += means[comp]
        np.rint(vals, out=vals)
        np.clip(vals, 0.0, 255.0, out=vals)
        out[c0:c1] = vals.astype(np.uint8)
    return out


def nbody(n: int, seed: int = SEED_NBODY):
    """Return (x, v, a): float32 [n, 4] arrays; x = (pos, mass), v = a = 0."""
    rng = _rng(seed)
    pos = rng.random((n, 3)).astype(np.float32)
    mass = rng.uniform(0.5, 1.0, size=n).astype(np.float32)
    x = np.zeros((n, 4), dtype=np.float32)
    x[:, :3] = pos
    x[:, 3] = mass
    v = np.zeros((n, 4), dtype=np.float32)
    a = np.zeros((n, 4), dtype=np.float32)
    return x, v, a


def fft_signals(nfft: int, n: int, seed: int = SEED_FFT) -> np.ndarray:
    """Complex64 array of shape (nfft, n), real and imaginary parts uniform in [-1, 1)."""
    rng = _rng(seed)
    re = rng.uniform(-1.0, 1.0, size=(nfft, n)).astype(np.float32)
    im = rng.uniform(-1.0, 1.0, size=(nfft, n)).astype(np.float32)
    out = np.empty((nfft, n), dtype=np.complex64)
    out.real = re
    out.imag = im
    return out


def round_up(v: int, m: int) -> int:
    return (v + m - 1) // m * m


def batch_shapes(n: int, seed: int = SEED_BATCH, lo: int = 64, hi: int = 2048) -> np.ndarray:
    """(n, 2) int64 array of (W, H), each side log-uniform in [lo, hi]."""
    u = _rng(seed).uniform(math.log(lo), math.log(hi), size=(n, 2))
    s = np.rint(np.exp(u)).astype(np.int64)
    return np.clip(s, lo, hi)


def batch_descriptors(shapes: np.ndarray, align: int = 256) -> tuple[np.ndarray, int]:
    """Descriptor table (n, 5) int64 of {offset, W, H, pitch, seed} and arena bytes.

    pitch = W rounded up to 16 bytes; every instance starts on an `align`-byte
    boundary; instance i's noise seed is 2 + i.
    """
    n = shapes.shape[0]
    desc = np.zeros((n, 5), dtype=np.int64)
    off = 0
    for i in range(n):
        w, h = int(shapes[i, 0]), int(shapes[i, 1])
        pitch = round_up(w, 16)
        desc[i] = (off, w, h, pitch, SEED_NOISE + i)
        off = round_up(off + pitch * h, align)
    return desc, off


def batch_instance(i: int, w: int, h: int, seed: int = SEED_BATCH) -> np.ndarray:
    """Pixels of instance i of a batch: (h, w) uint8 from its own PCG64 stream."""
    return _rng(seed * 1_000_000 + i).integers(0, 256, size=(h, w), dtype=np.uint8)


def batch_arena(desc: np.ndarray, nbytes: int, seed: int = SEED_BATCH, out: np.ndarray | None = None,
                indices=None) -> np.ndarray:
    """Fill a uint8 arena with each instance's pixels (padding bytes are 0)."""
    if out is None:
        out = np.zeros(nbytes, dtype=np.uint8)
    idx = range(desc.shape[0]) if indices is None else indices
    for i in idx:
        off, w, h, pitch, _ = (int(t) for t in desc[i])
        view = out[off:off + h * pitch].reshape(h, pitch)
        view[:, :w] = batch_instance(i, w, h, seed)
    return out


def instance_view(arena: np.ndarray, desc_row) -> np.ndarray:
    """(H, W) view of one instance inside an arena."""
    off, w, h, pitch, _ = (int(t) for t in desc_row)
    return arena[off:off + h * pitch].reshape(h, pitch)[:, :w]


# ----------------------------------------------------------------------------------------------
# Random compound skeletons for the cost model: a stage list drawn from the built-in library,
# a skeleton kind and an element count. Only the description is drawn here.
# ----------------------------------------------------------------------------------------------
IMAGE_STAGE_NAMES = ("noise", "solarise", "mirror", "threshold3", "blur5")


def random_skeletons(n: int, seed: int = SEED_MODEL, min_log2: int = 12, max_log2: int = 28):
    """List of dicts {kind, stages, width, rows, seed} describing random u8/f32 skeletons.

    kind is one of 'pipeline', 'map', 'mapreduce', 'saxpy'; image skeletons have 1..6 stages;
    the element count is 2**U(min_log2, max_log2) split into rows of a random power-of-two width.
    """
    rng = _rng(seed)
    out = []
    for _ in range(n):
        kind = ("pipeline", "map", "mapreduce", "saxpy")[int(rng.integers(0, 4))]
        log2n = float(rng.uniform(min_log2, max_log2))
        total = int(2 ** log2n)
        if kind == "saxpy":
            out.append({"kind": kind, "stages": ["saxpy"], "width": total, "rows": 1, "seed": 0})
            continue
        k = int(rng.integers(1, 7))
        stages = [IMAGE_STAGE_NAMES[int(t)] for t in rng.integers(0, 4, size=k)]
        if kind == "mapreduce":
            stages[-1] = "threshold3"
        if rng.random() < 0.3 and kind != "mapreduce":
            stages.insert(int(rng.integers(0, len(stages) + 1)), "blur5")
        lw = int(rng.integers(6, 14))
        width = min(1 << lw, total)
        width += int(rng.integers(0, 16)) if rng.random() < 0.25 else 0
        rows = max(1, total // width)
        out.append({"kind": kind, "stages": stages, "width": width, "rows": rows,
                    "seed": int(rng.integers(0, 2 ** 31))})
    return out
