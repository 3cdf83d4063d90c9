"""Pins of the image-stage oracle against facts fixed outside it (no GPU)."""
import os

import numpy as np
import pytest

from oracle import image as O
from paper_1510_06585_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rotl(x, r):
    return ((x << r) | (x >> (32 - r))) & 0xFFFFFFFF


def _murmur3_x86_32(data: bytes, seed: int) -> int:
    """Body and tail of MurmurHash3_x86_32; the finaliser is the oracle's fmix32."""
    c1, c2 = 0xCC9E2D51, 0x1B873593
    h = seed
    nblocks = len(data) // 4
    for i in range(nblocks):
        k = int.from_bytes(data[4 * i:4 * i + 4], "little")
        k = _rotl((k * c1) & 0xFFFFFFFF, 15)
        h ^= (k * c2) & 0xFFFFFFFF
        h = (_rotl(h, 13) * 5 + 0xE6546B64) & 0xFFFFFFFF
    tail = data[4 * nblocks:]
    k = 0
    for j in reversed(range(len(tail))):
        k ^= tail[j] << (8 * j)
    if tail:
        k = _rotl((k * c1) & 0xFFFFFFFF, 15)
        h ^= (k * c2) & 0xFFFFFFFF
    h ^= len(data)
    return int(O.fmix32(h))


def test_fmix32_matches_published_murmur3_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "murmur3_x86_32_vectors.txt")) if l.strip()
            and not l.startswith("#")]
    assert len(rows) == 10
    for data_hex, seed_hex, want_hex in rows:
        data = b"" if data_hex == "-" else bytes.fromhex(data_hex)
        assert _murmur3_x86_32(data, int(seed_hex, 16)) == int(want_hex, 16), data


def test_hash32_is_uint32_and_chains_seed_x_y():
    # empty-input MurmurHash3 with seed s is F(s): chain three of them as the definition states
    s, x, y = 2, 77, 1023
    want = _murmur3_x86_32(b"", _murmur3_x86_32(b"", _murmur3_x86_32(b"", s) ^ x) ^ y)
    assert int(O.hash32(s, x, y)) == want
    assert int(O.hash32(s, x, y)) != int(O.hash32(s, y, x))
    h = O.hash32(7, np.arange(1000)[None, :], np.arange(50)[:, None])
    assert h.max() < 2 ** 32 and h.dtype == np.uint64


def test_noise_offsets_are_uniform_on_minus20_to_20():
    img = np.full((200, 205), 128, dtype=np.uint8)  # no clamping possible
    d = O.noise(img, seed=2).astype(np.int64) - 128
    assert d.min() >= -20 and d.max() <= 20
    counts = np.bincount(d.reshape(-1) + 20, minlength=41)
    assert counts.shape == (41,) and counts.min() > 0
    expected = d.size / 41
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 90.0  # 40 degrees of freedom; p ~ 1e-5 at 90


def test_noise_clamps_at_both_ends():
    lo = O.noise(np.zeros((64, 64), np.uint8), seed=9)
    hi = O.noise(np.full((64, 64), 255, np.uint8), seed=9)
    assert lo.max() <= 20 and hi.min() >= 235
    # a draw of n <= 0 clamps to 0: about 21 of 41 outcomes
    frac0 = (lo == 0).mean()
    assert abs(frac0 - 21 / 41) < 0.03
    frac255 = (hi == 255).mean()
    assert abs(frac255 - 21 / 41) < 0.03


def test_noise_uses_global_coordinates_of_its_partition():
    img = inputs.filter_image(40, 56, seed=11)
    full = O.noise(img, seed=5)
    part = O.noise(img[10:30, 16:40], seed=5, x0=16, y0=10)
    assert np.array_equal(full[10:30, 16:40], part)
    assert not np.array_equal(O.noise(img[10:30, 16:40], seed=5), part)


def test_solarise_identity_below_128_and_symmetric():
    p = np.arange(256, dtype=np.uint8)
    s = O.solarise(p).astype(np.int64)
    assert np.array_equal(s[:128], np.arange(128))            # identity on [0, 127]
    assert np.array_equal(s, s[::-1])                        # sol(p) == sol(255 - p)
    assert s.max() == 127 and s[255] == 0 and s[128] == 127


def test_mirror_is_fliplr_and_an_involution():
    img = inputs.filter_image(17, 33, seed=3)
    assert np.array_equal(O.mirror(img), np.fliplr(img))
    assert np.array_equal(O.mirror(O.mirror(img)), img)
    ramp = np.tile(np.arange(10, dtype=np.uint8), (3, 1))
    assert np.array_equal(O.mirror(ramp)[0], np.arange(9, -1, -1))
    vol = inputs.volume(3, 4, 5, seed=1)
    assert np.array_equal(O.mirror(vol), vol[:, :, ::-1])


def _blur_brute(img):
    h, w = img.shape
    out = np.zeros_like(img)
    for y in range(h):
        for x in range(w):
            s = 0
            for dy in range(-2, 3):
                for dx in range(-2, 3):
                    yy = min(max(y + dy, 0), h - 1)
                    xx = min(max(x + dx, 0), w - 1)
                    s += int(img[yy, xx])
            out[y, x] = (s + 12) // 25
    return out


def test_blur_brute_force_8x8_and_small_shapes():
    for (h, w) in [(8, 8), (1, 1), (1, 7), (5, 1), (3, 9), (8, 13)]:
        img = inputs.filter_image(h, w, seed=h * 100 + w)
        assert np.array_equal(O.blur5(img), _blur_brute(img)), (h, w)


def test_blur_matches_scipy_correlate_sum():
    ndimage = pytest.importorskip("scipy.ndimage")
    img = inputs.filter_image(37, 50, seed=4)
    s = ndimage.correlate(img.astype(np.int64), np.ones((5, 5), np.int64), mode="nearest")
    assert np.array_equal(O.blur5(img), ((s + 12) // 25).astype(np.uint8))


def test_blur_fixed_point_and_commutes_with_mirror():
    c = np.full((9, 11), 77, np.uint8)
    assert np.array_equal(O.blur5(c), c)
    img = inputs.filter_image(20, 23, seed=8)
    assert np.array_equal(O.blur5(O.mirror(img)), O.mirror(O.blur5(img)))
    vol = inputs.volume(3, 10, 12, seed=2)
    assert np.array_equal(O.blur5(vol)[1], O.blur5(vol[1]))  # per plane


def test_threshold_ties_and_counts_match_histogram():
    p = np.array([0, 84, 85, 86, 169, 170, 171, 255], np.uint8)
    assert list(O.threshold3(p)) == [0, 0, 1, 1, 1, 2, 2, 2]
    vol = inputs.volume(4, 33, 35, seed=3)
    labels, counts = O.segmentation(vol)
    hist, _ = np.histogram(vol, bins=[0, 85, 170, 256])
    assert np.array_equal(counts, hist.astype(np.int64))
    assert np.array_equal(counts, np.bincount(labels.reshape(-1), minlength=3))
    assert counts.sum() == vol.size and counts.dtype == np.int64


def _pipeline_brute(img, seed):
    """Per-pixel formula of noise -> solarise -> mirror: out[y][x] takes source column W-1-x."""
    h, w = img.shape
    out = np.zeros_like(img)
    for y in range(h):
        for x in range(w):
            xs = w - 1 - x
            hv = int(O.hash32(seed, xs, y))
            p = min(max(int(img[y, xs]) + hv % 41 - 20, 0), 255)
            out[y, x] = p if p < 128 else 255 - p
    return out


def test_filter_pipeline_brute_force_8x8_and_odd_widths():
    for (h, w) in [(8, 8)] + [(3, k) for k in range(1, 34, 4)]:
        img = inputs.filter_image(h, w, seed=w)
        assert np.array_equal(O.filter_pipeline(img, 2), _pipeline_brute(img, 2)), (h, w)


def test_noise_then_solarise_exhaustive_table():
    # every (pixel, noise offset) pair: clamp then fold at 128
    p = np.repeat(np.arange(256), 41)
    n = np.tile(np.arange(-20, 21), 256)
    q = np.clip(p + n, 0, 255)
    folded = np.minimum(q, 255 - q)  # equals solarise for all q in [0, 255]
    assert np.array_equal(O.solarise(q.astype(np.uint8)).astype(np.int64), folded)
