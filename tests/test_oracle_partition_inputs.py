"""Pins of the partition-constraint checker and the seeded generators (no GPU)."""
import numpy as np

from oracle import partition as P
from paper_1510_06585_gb300 import inputs


def test_partition_checker_accepts_valid_and_flags_each_violation():
    assert P.check_plan(1024, [(0, 512), (512, 512)], epu=64, nu=2, block=32) == []
    assert P.check_plan(100, [(0, 64), (64, 36)], epu=4, nu=2) == []
    assert any("multiple of nu" in e for e in P.check_plan(64, [(0, 64)], epu=3, nu=2))
    assert any("gap or overlap" in e for e in P.check_plan(64, [(0, 30), (32, 32)], epu=2, nu=1))
    assert any("whole number" in e for e in P.check_plan(64, [(0, 30), (30, 34)], epu=4, nu=1))
    assert any("cover" in e for e in P.check_plan(64, [(0, 32)], epu=4, nu=1))
    assert any("block size" in e for e in P.check_plan(256, [(0, 96), (96, 160)], epu=2, nu=1, block=64))


def test_generators_are_deterministic_and_shaped():
    a = inputs.filter_image(32, 48)
    assert a.dtype == np.uint8 and a.shape == (32, 48)
    assert np.array_equal(a, inputs.filter_image(32, 48))
    v = inputs.volume(20, 8, 8)
    assert v.dtype == np.uint8 and v.shape == (20, 8, 8)
    # chunk-wise seeding: a leading sub-volume is a prefix of the bigger one
    assert np.array_equal(inputs.volume(16, 8, 8), v[:16])
    x, vv, aa = inputs.nbody(100)
    assert x.dtype == np.float32 and x.shape == (100, 4)
    assert (x[:, :3] >= 0).all() and (x[:, :3] < 1).all()
    assert (x[:, 3] >= 0.5).all() and (x[:, 3] <= 1).all()
    assert not vv.any() and not aa.any()


def test_volume_mixture_statistics():
    v = inputs.volume(16, 64, 64).astype(np.float64)
    hist, _ = np.histogram(v, bins=[0, 85, 170, 256])
    assert np.allclose(hist / v.size, 1 / 3, atol=0.01)
    assert abs(v[v < 85].mean() - 40) < 1 and abs(v[v >= 170].mean() - 220) < 1


def test_batch_descriptors_alignment_and_ranges():
    shapes = inputs.batch_shapes(512)
    assert shapes.min() >= 64 and shapes.max() <= 2048
    desc, nbytes = inputs.batch_descriptors(shapes)
    assert (desc[:, 0] % 256 == 0).all() and (desc[:, 3] % 16 == 0).all()
    assert (desc[:, 3] >= desc[:, 1]).all()
    ends = desc[:, 0] + desc[:, 2] * desc[:, 3]
    assert (ends[:-1] <= desc[1:, 0]).all() and ends[-1] <= nbytes
    arena = inputs.batch_arena(desc[:4], int(ends[3]))
    img = inputs.instance_view(arena, desc[2])
    assert img.shape == (desc[2, 2], desc[2, 1])
    # log-uniform sides: the median side is near sqrt(64 * 2048)
    assert 250 < np.median(shapes) < 470


def test_random_skeletons_shapes():
    sk = inputs.random_skeletons(200)
    assert len(sk) == 200
    for s in sk:
        assert 1 <= len(s["stages"]) <= 7
        assert s["width"] >= 1 and s["rows"] >= 1
        if s["kind"] == "mapreduce":
            assert s["stages"][-1] == "threshold3"
