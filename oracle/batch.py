"""Whole-batch oracle check of the batched Filter Pipeline + blur — test infrastructure only (see
``oracle/__init__``).

The batched workload (thousands of independent skeleton instances of uneven sizes in one launch)
is checked instance by instance against the single-instance oracle: instance i is regenerated from
its own seeded stream, run through noise (its own seed), solarise, mirror and the 5x5 blur
(``oracle.image.filter_blur_pipeline``), and reduced to a 64-bit BLAKE2b digest of its bytes, so
that a pool of worker processes can cover a 1.3 G-pixel batch without moving pixels between
processes. Parity is pinned by tests/test_oracle_batch.py (the digests equal those of the
instances evaluated in full through ``oracle.skeleton``).
"""
from __future__ import annotations

import hashlib
import multiprocessing as mp

import numpy as np

from paper_1510_06585_gb300 import inputs

from . import image


def digest(img: np.ndarray) -> bytes:
    """64-bit BLAKE2b digest of an (H, W) uint8 image's bytes, row by row."""
    return hashlib.blake2b(np.ascontiguousarray(img).tobytes(), digest_size=8).digest()


def instance_digest(job) -> tuple[int, bytes]:
    """job = (i, W, H, noise_seed): the digest of instance i's Filter Pipeline + blur output."""
    i, w, h, seed = (int(v) for v in job)
    img = inputs.batch_instance(i, w, h)
    return i, digest(image.filter_blur_pipeline(img, seed))


def batch_digests(desc: np.ndarray, processes: int = 1) -> list[bytes]:
    """Digests of every instance of a batch described by `desc` (rows {offset, W, H, pitch, seed}).
    Worker processes are spawned (never forked: the caller may hold a CUDA context)."""
    jobs = [(i, int(desc[i, 1]), int(desc[i, 2]), int(desc[i, 4])) for i in range(desc.shape[0])]
    # largest first, so that the pool's tail is short
    jobs.sort(key=lambda j: -j[1] * j[2])
    out: list[bytes | None] = [None] * len(jobs)
    if processes <= 1:
        for j in jobs:
            i, d = instance_digest(j)
            out[i] = d
    else:
        with mp.get_context("spawn").Pool(processes) as pool:
            for i, d in pool.imap_unordered(instance_digest, jobs, chunksize=4):
                out[i] = d
    return out  # type: ignore[return-value]
