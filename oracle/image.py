"""Oracle for the image skeleton stages — test infrastructure only (see ``oracle/__init__``).

Each stage materialises its whole output, exactly as a kernel-per-stage
execution would; nothing is fused or reordered.

Paper references (Section 4, benchmark descriptions): the Filter Pipeline
composes a noise filter, Solarize and Mirror, each applicable line by line;
Segmentation maps a 3-D greyscale volume to three classes (white / grey /
black). The executor's workloads fix the concrete formulas the paper leaves
open (it names the filters, not their arithmetic):

* noise     : p' = clamp(p + (hash32(seed, x, y) mod 41) - 20, 0, 255), with
              hash32(s, x, y) = F(F(F(s) ^ x) ^ y) and F the 32-bit MurmurHash3
              finaliser (Appleby, public domain); x = column and y = row of the
              stage's input in global coordinates (the paper's Offset trait,
              Section 3.4), rows of a volume counted across planes.
* solarise  : p < 128 ? p : 255 - p.
* mirror    : left-right flip of every row, out[y][x] = in[y][W-1-x].
* blur5     : 5x5 box filter per plane, edge pixels replicated,
              out = (sum of the 25 pixels + 12) // 25 (round half up).
* threshold3: label = (p >= 85) + (p >= 170)  (ties go to the upper class).
* counts    : int64 histogram of the labels.

Pins (tests/test_oracle_image.py): F against published MurmurHash3 test
vectors; solarise by its symmetry and identity properties; mirror against
numpy.fliplr and the involution property; blur against an explicit 25-term
loop and scipy's correlate; threshold/counts against numpy.histogram; the
composed pipeline against a per-pixel brute force on 8x8.
"""
from __future__ import annotations

import numpy as np

_M32 = np.uint64(0xFFFFFFFF)


def fmix32(h):
    """MurmurHash3 32-bit finaliser on uint32 values (array or scalar), wrapping mod 2^32."""
    h = np.asarray(h, dtype=np.uint64) & _M32
    h = h ^ (h >> np.uint64(16))
    h = (h * np.uint64(0x85EBCA6B)) & _M32
    h = h ^ (h >> np.uint64(13))
    h = (h * np.uint64(0xC2B2AE35)) & _M32
    h = h ^ (h >> np.uint64(16))
    return h


def hash32(seed, x, y):
    """hash32(seed, x, y) = F(F(F(seed) ^ x) ^ y), all uint32."""
    s = np.asarray(seed, dtype=np.uint64) & _M32
    xx = np.asarray(x, dtype=np.uint64) & _M32
    yy = np.asarray(y, dtype=np.uint64) & _M32
    return fmix32(fmix32(fmix32(s) ^ xx) ^ yy)


def _rows(img: np.ndarray) -> np.ndarray:
    """View an (H, W) image or (D, H, W) volume as (rows, W)."""
    return img.reshape(-1, img.shape[-1])


def noise(img: np.ndarray, seed: int, x0: int = 0, y0: int = 0) -> np.ndarray:
    """Noise stage. (x0, y0) is the global offset of this partition (Offset trait)."""
    r = _rows(img)
    rows, w = r.shape
    ys = (np.arange(rows, dtype=np.uint64) + np.uint64(y0))[:, None]
    xs = (np.arange(w, dtype=np.uint64) + np.uint64(x0))[None, :]
    h = hash32(seed, xs, ys)
    n = (h % np.uint64(41)).astype(np.int64) - 20
    out = np.clip(r.astype(np.int64) + n, 0, 255).astype(np.uint8)
    return out.reshape(img.shape)


def solarise(img: np.ndarray) -> np.ndarray:
    p = img.astype(np.int64)
    return np.where(p < 128, p, 255 - p).astype(np.uint8)


def mirror(img: np.ndarray) -> np.ndarray:
    """Horizontal (left-right) mirror of every row."""
    return np.ascontiguousarray(img[..., ::-1])


def blur5(img: np.ndarray) -> np.ndarray:
    """5x5 box blur of each plane with replicated edges, (sum + 12) // 25."""
    planes = img.reshape(-1, img.shape[-2], img.shape[-1]) if img.ndim >= 2 else img[None, None, :]
    out = np.empty_like(planes)
    for k in range(planes.shape[0]):
        p = np.pad(planes[k].astype(np.int64), 2, mode="edge")
        h, w = planes[k].shape
        s = np.zeros((h, w), dtype=np.int64)
        for dy in range(5):
            for dx in range(5):
                s += p[dy:dy + h, dx:dx + w]
        out[k] = ((s + 12) // 25).astype(np.uint8)
    return out.reshape(img.shape)


def threshold3(img: np.ndarray) -> np.ndarray:
    p = img.astype(np.int64)
    return ((p >= 85).astype(np.int64) + (p >= 170).astype(np.int64)).astype(np.uint8)


def class_counts(labels: np.ndarray, k: int = 3) -> np.ndarray:
    """counts[c] = number of elements equal to c, as int64."""
    flat = labels.reshape(-1)
    return np.array([int(np.count_nonzero(flat == c)) for c in range(k)], dtype=np.int64)


def value_sum(img: np.ndarray) -> np.ndarray:
    """Sum of all values as a one-element int64 array (MapReduce + over a non-classifying stage)."""
    return np.array([int(img.astype(np.int64).sum())], dtype=np.int64)


STAGES = {
    "noise": noise,
    "solarise": solarise,
    "mirror": mirror,
    "blur5": blur5,
    "threshold3": threshold3,
}


def apply_stage(name: str, img: np.ndarray, seed: int = 0, x0: int = 0, y0: int = 0) -> np.ndarray:
    if name == "noise":
        return noise(img, seed, x0, y0)
    return STAGES[name](img)


def filter_pipeline(img: np.ndarray, seed: int) -> np.ndarray:
    """Filter Pipeline of Section 4: noise, then solarise, then mirror."""
    return mirror(solarise(noise(img, seed)))


def filter_blur_pipeline(img: np.ndarray, seed: int) -> np.ndarray:
    """Filter Pipeline followed by the 5x5 box blur (the batched workload's instance)."""
    return blur5(filter_pipeline(img, seed))


def segmentation(vol: np.ndarray):
    """Map (threshold into 3 classes) then MapReduce (+) of the class counts."""
    labels = threshold3(vol)
    return labels, class_counts(labels, 3)
