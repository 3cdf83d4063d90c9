"""Pins of the depth-first skeleton evaluator (no GPU)."""
import numpy as np

from oracle import image as I
from oracle import nbody as N
from oracle import skeleton as S
from paper_1510_06585_gb300 import inputs


def st(name, **p):
    return ("stage", name, p)


def test_pipeline_runs_stages_in_order():
    img = inputs.filter_image(16, 24, seed=1)
    out, _ = S.evaluate_image(("pipeline", [st("noise", seed=3), st("solarise")]), img)
    assert np.array_equal(out, I.solarise(I.noise(img, 3)))
    assert not np.array_equal(out, I.noise(I.solarise(img), 3))


def test_depth_first_order_of_pipeline_loop_pipeline():
    # pipeline(K1, loop(K2), K3) runs K1, K2 k times, then K3
    trace = []
    tree = ("pipeline", [st("noise", seed=1), ("loop", st("mirror"), 3), st("solarise")])
    S.evaluate_image(tree, inputs.filter_image(4, 4), trace)
    assert trace == ["noise", "mirror", "mirror", "mirror", "solarise"]


def test_loop_of_even_mirrors_is_identity():
    img = inputs.filter_image(5, 9, seed=2)
    out, _ = S.evaluate_image(("loop", st("mirror"), 4), img)
    assert np.array_equal(out, img)


def test_map_over_planes_equals_whole_volume_for_pointwise_stages():
    vol = inputs.volume(5, 7, 9, seed=4)
    body = ("pipeline", [st("noise", seed=8), st("solarise"), st("mirror")])
    out, _ = S.evaluate_image(("map", body), vol)
    whole = I.mirror(I.solarise(I.noise(vol, 8)))
    assert np.array_equal(out, whole)


def test_map_with_blur_is_per_plane():
    vol = inputs.volume(3, 8, 10, seed=5)
    out, _ = S.evaluate_image(("map", st("blur5")), vol)
    for k in range(3):
        assert np.array_equal(out[k], I.blur5(vol[k]))


def test_mapreduce_counts_match_histogram():
    vol = inputs.volume(3, 20, 21, seed=6)
    labels, counts = S.evaluate_image(("mapreduce", st("threshold3"), "add"), vol)
    hist, _ = np.histogram(vol, bins=[0, 85, 170, 256])
    assert np.array_equal(counts, hist)
    assert np.array_equal(labels, I.threshold3(vol))
    _, total = S.evaluate_image(("mapreduce", st("solarise"), "add"), vol)
    assert total[0] == int(I.solarise(vol).astype(np.int64).sum())


def test_nbody_tree_is_accel_then_loop():
    x, v, a = inputs.nbody(32, seed=9)
    p = {"G": 1 / 32, "eps": 1e-3, "dt": 1e-3}
    trace = []
    state = (x.astype(np.float64), np.zeros((32, 3)), np.zeros((32, 3)))
    got = S.evaluate_nbody(("pipeline", [st("nbody_accel", **p), ("loop", st("nbody_kdk", **p), 5)]), state, trace)
    want = N.simulate(x, 5)
    assert trace == ["nbody_accel"] + ["nbody_kdk"] * 5
    for g, w in zip(got, want):
        assert np.array_equal(np.asarray(g)[:, :3], np.asarray(w)[:, :3])


def test_loop_while_changed_stops_at_the_fixed_point():
    img = inputs.filter_image(16, 16, seed=16)
    trace = []
    out, _ = S.evaluate_image(("loop_while", st("blur5"), 1000), img, trace)
    assert np.array_equal(I.blur5(out), out)          # a fixed point of the body
    n = len(trace)                                    # run n made no change, run n - 1 did
    prev = img
    for _ in range(n - 2):
        prev = I.blur5(prev)
    assert not np.array_equal(I.blur5(prev), prev)
    assert np.array_equal(I.blur5(I.blur5(prev)), I.blur5(prev))
    capped, _ = S.evaluate_image(("loop_while", st("blur5"), 3), img)
    assert np.array_equal(capped, I.blur5(I.blur5(I.blur5(img))))
    # an idempotent body stops after its second run
    t2 = []
    S.evaluate_image(("loop_while", st("solarise"), 50), img, t2)
    assert len(t2) == 2
