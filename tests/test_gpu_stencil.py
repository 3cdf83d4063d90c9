"""GPU parity of the TMA-staged stencil groups (5x5 box blur fused with pointwise prefixes and
suffixes) and of batched execution, against the CPU oracle: bit-exact."""
import ctypes
import os

import numpy as np
import pytest
import torch

from gpu_util import build_image_tree, oracle_tree, run_image
from oracle import image as O
from oracle import batch as OB
from oracle import skeleton as S
from paper_1510_06585_gb300 import inputs
from paper_1510_06585_gb300 import mrw as M

pytestmark = pytest.mark.gpu

FILTER_BLUR = ["noise", "solarise", "mirror", "blur5"]


def test_blur_alone_on_edge_shapes():
    tree = M.pipeline(M.stage("blur5"))
    for (h, w) in [(1, 1), (1, 7), (5, 1), (8, 8), (2, 2), (33, 47), (300, 333), (1024, 1024), (40, 1000)]:
        img = inputs.filter_image(h, w, seed=h + 7 * w)
        got, _ = run_image(tree, img)
        assert np.array_equal(got, O.blur5(img)), (h, w)


@pytest.mark.parametrize("names", [
    FILTER_BLUR,
    ["mirror", "blur5"],
    ["blur5", "mirror"],
    ["noise", "mirror", "blur5", "noise", "mirror", "solarise"],
    ["blur5", "noise", "blur5"],
    ["mirror", "mirror", "noise", "blur5", "mirror", "threshold3"],
    ["noise", "noise", "noise", "blur5"],
])
def test_stencil_prefix_suffix_orders(names):
    seeds = {i: 1000 + 17 * i for i in range(len(names))}
    tree = build_image_tree(names, seeds)
    for (h, w) in [(8, 8), (37, 129), (130, 250), (3, 17)]:
        img = inputs.filter_image(h, w, seed=h * w)
        want, _ = S.evaluate_image(oracle_tree(names, seeds), img)
        for cfg in (M.config(), M.config(tile_rows=16, tile_cols=64, ctas_per_sm=2),
                    M.config(fusion=M.MRW_FUSE_NONE)):
            got, _ = run_image(tree, img, cfg)
            assert np.array_equal(got, want), (names, h, w, cfg.as_tuple())


@pytest.mark.parametrize("names", [
    FILTER_BLUR,
    ["noise", "mirror", "noise", "solarise", "blur5"],
    ["threshold3", "mirror", "blur5"],
    # each prefix sequence the kernel runs without walking the op list, and near misses of them
    ["noise", "blur5"],
    ["solarise", "mirror", "blur5"],
    ["mirror", "noise", "mirror", "solarise", "blur5"],
    ["solarise", "noise", "blur5"],
    ["noise", "solarise", "solarise", "blur5"],
])
def test_row_streaming_blur_strip_and_segment_edges(names):
    # blur groups with only a prefix run on the row-streaming kernel: strips of 124 output columns,
    # items of 4 x tile_rows rows streamed through 8-row TMA boxes; the shapes put image edges on,
    # just before and just after strip and item boundaries (tile_rows 2 -> 8-row items, one box each)
    seeds = {i: 300 + 11 * i for i in range(len(names))}
    tree = build_image_tree(names, seeds)
    otree = oracle_tree(names, seeds)
    for (h, w) in [(129, 124), (127, 125), (64, 123), (65, 248), (200, 249), (257, 372), (6, 4), (4, 6), (9, 130)]:
        img = inputs.filter_image(h, w, seed=h + w)
        want, _ = S.evaluate_image(otree, img)
        for cfg in (M.config(), M.config(tile_rows=16), M.config(tile_rows=2, ctas_per_sm=2)):
            got, _ = run_image(tree, img, cfg)
            assert np.array_equal(got, want), (names, h, w, cfg.as_tuple())
        got, _ = run_image(tree, img, pitch=w + 16 * 9 - w % 16)  # a wider row pitch than needed
        assert np.array_equal(got, want), (names, h, w, "pitch")


def test_every_candidate_tile_shape():
    img = inputs.filter_image(200, 453, seed=9)
    tree = build_image_tree(FILTER_BLUR, {0: 2})
    want = O.filter_blur_pipeline(img, 2)
    for c in M.tune_candidates(tree, [img, img]):
        got, _ = run_image(tree, img, c)
        assert np.array_equal(got, want), c.as_tuple()


def test_map_blur_is_per_plane_on_volumes():
    vol = inputs.volume(3, 20, 50, seed=1)
    tree = M.map_(build_image_tree(["noise", "blur5"], {0: 4}))
    got, _ = run_image(tree, vol)
    want, _ = S.evaluate_image(("map", oracle_tree(["noise", "blur5"], {0: 4})), vol)
    assert np.array_equal(got, want)


def _batch(shapes):
    desc, nbytes = inputs.batch_descriptors(shapes)
    arena = inputs.batch_arena(desc, nbytes)
    return desc, nbytes, arena


def _check_instances(out_arena, in_arena, desc, idx, names=FILTER_BLUR):
    for i in idx:
        img = inputs.instance_view(in_arena, desc[i])
        seed = int(desc[i, 4])
        want, _ = S.evaluate_image(oracle_tree(names, {0: seed}), img)
        got = inputs.instance_view(out_arena, desc[i])
        assert np.array_equal(got, want), (i, desc[i])


def test_batched_small_uneven_instances():
    rng = np.random.Generator(np.random.PCG64(3))
    shapes = np.stack([rng.integers(1, 300, size=60), rng.integers(1, 200, size=60)], axis=1)
    shapes[:4] = [[1, 1], [16, 1], [1, 16], [17, 3]]
    desc, nbytes, arena = _batch(shapes)
    tree = M.map_(build_image_tree(FILTER_BLUR))  # stage seed 0: each instance's seed applies
    x = torch.from_numpy(arena).cuda()
    for cfg in (None, M.config(tile_rows=16, tile_cols=64), M.config(fusion=M.MRW_FUSE_NONE)):
        y = torch.zeros_like(x)
        M.execute_batched(tree, x, y, desc, cfg).wait(60000)
        _check_instances(y.cpu().numpy(), arena, desc, range(len(desc)))
    # pointwise-only batched trees run through the same persistent kernel
    tree2 = M.map_(build_image_tree(["noise", "mirror"]))
    y = torch.zeros_like(x)
    M.execute_batched(tree2, x, y, desc).wait(60000)
    _check_instances(y.cpu().numpy(), arena, desc, range(len(desc)), ["noise", "mirror"])


def test_batched_4096_log_uniform_full_size():
    shapes = inputs.batch_shapes(4096)
    desc, nbytes, arena = _batch(shapes)
    tree = M.map_(build_image_tree(FILTER_BLUR))
    x = torch.from_numpy(arena).cuda()
    y = torch.zeros_like(x)
    f = M.execute_batched(tree, x, y, desc)
    f.wait(120000)
    out = y.cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(11))
    idx = set(rng.choice(4096, size=40, replace=False).tolist())
    idx |= {int(np.argmin(shapes.prod(axis=1))), int(np.argmax(shapes.prod(axis=1))), 0, 4095}
    _check_instances(out, arena, desc, sorted(idx))
    # every instance: the oracle's output digests (computed by a pool of spawned processes from the
    # seeded inputs) against the digests of the executor's output
    want = OB.batch_digests(desc, processes=max(1, min(16, os.cpu_count() or 1)))
    got = [OB.digest(inputs.instance_view(out, desc[i])) for i in range(len(desc))]
    bad = [i for i in range(len(desc)) if got[i] != want[i]]
    assert not bad, (len(bad), bad[:10])
    # a second launch of the cached graph gives the same bytes
    y2 = torch.zeros_like(x)
    M.execute_batched(tree, x, y2, desc).wait(120000)
    assert torch.equal(y, y2)


def test_batched_rejects_bad_descriptors():
    desc, nbytes, arena = _batch(np.array([[20, 10], [30, 5]]))
    x = torch.from_numpy(arena).cuda()
    y = torch.zeros_like(x)
    tree = M.map_(build_image_tree(FILTER_BLUR))
    bad = desc.copy()
    bad[1, 3] = 24  # pitch not a multiple of 16
    with pytest.raises(M.MrwError) as e:
        M.execute_batched(tree, x, y, bad)
    assert e.value.status == M.MRW_ERR_CONSTRAINT
    bad = desc.copy()
    bad[1, 0] = nbytes  # outside the arena
    with pytest.raises(M.MrwError) as e:
        M.execute_batched(tree, x, y, bad)
    assert e.value.status == M.MRW_ERR_SHAPE


@pytest.mark.parametrize("shape", [(16, 16), (64, 64), (100, 137), (3, 40)])
def test_blur_until_fixed_point_is_decided_on_the_device(shape):
    img = inputs.filter_image(*shape, seed=shape[0])
    tree = M.loop(M.stage("blur5"), 1000, M.MRW_LOOP_WHILE_CHANGED)
    want, _ = S.evaluate_image(("loop_while", ("stage", "blur5", {}), 1000), img)
    for cfg in (None, M.config(tile_rows=16, tile_cols=64)):
        got, _ = run_image(tree, img, cfg)
        assert np.array_equal(got, want), shape
    assert np.array_equal(O.blur5(want), want)


def test_while_loop_inside_a_pipeline_and_capped_bodies():
    img = inputs.filter_image(70, 90, seed=4)
    body = M.pipeline(M.stage("mirror"), M.stage("blur5"), M.stage("noise", seed=3), M.stage("blur5"))
    for cap in (1, 7, 400):
        tree = M.pipeline(M.stage("noise", seed=9), M.loop(body, cap, M.MRW_LOOP_WHILE_CHANGED),
                          M.stage("solarise"))
        otree = ("pipeline", [("stage", "noise", {"seed": 9}),
                              ("loop_while", ("pipeline", [("stage", "mirror", {}), ("stage", "blur5", {}),
                                                          ("stage", "noise", {"seed": 3}), ("stage", "blur5", {})]),
                               cap),
                              ("stage", "solarise", {})])
        want, _ = S.evaluate_image(otree, img)
        for cfg in (M.config(), M.config(fusion=M.MRW_FUSE_NONE)):
            for _ in range(2):  # the second run reuses the cached loop graph
                got, _ = run_image(tree, img, cfg)
                assert np.array_equal(got, want), (cap, cfg.as_tuple())
    # an idempotent pointwise body stops after its second run
    got, _ = run_image(M.loop(M.stage("solarise"), 50, M.MRW_LOOP_WHILE_CHANGED), img)
    assert np.array_equal(got, O.solarise(img))


def test_batched_plan_cache_eviction_under_concurrent_callers():
    # Four host threads, each on its own stream, run batched launches with 48 distinct descriptor
    # tables between them (more than the 32 cached plans): entries are evicted while other
    # threads hold and launch theirs. Every output must still be the oracle's.
    import threading

    from oracle import batch as OB
    lib = M.load()
    tree = M.map_(M.pipeline(M.stage("noise"), M.stage("solarise"), M.stage("mirror"), M.stage("blur5")))
    jobs = []
    for k in range(48):
        rng = np.random.Generator(np.random.PCG64(900 + k))
        shapes = np.stack([rng.integers(1, 70, size=3), rng.integers(1, 50, size=3)], axis=1)
        desc, nbytes = inputs.batch_descriptors(shapes)
        arena = inputs.batch_arena(desc, nbytes, seed=900 + k)
        want = [OB.digest(O.filter_blur_pipeline(inputs.instance_view(arena, d), int(d[4]))) for d in desc]
        jobs.append((np.ascontiguousarray(desc, dtype=np.int64), arena, want))
    errors = []

    def worker(tid):
        try:
            stream = torch.cuda.Stream()
            for rep in range(2):
                for k in range(tid, 48, 4):
                    desc, arena, want = jobs[k]
                    x = torch.from_numpy(arena).cuda()
                    y = torch.zeros_like(x)
                    torch.cuda.synchronize()
                    fut = ctypes.c_void_p()
                    st = lib.mrw_execute_batched(tree.h, x.data_ptr(), y.data_ptr(), x.numel(),
                                                 desc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                                 desc.shape[0], None, stream.cuda_stream, ctypes.byref(fut))
                    if st != M.MRW_OK:
                        errors.append((tid, k, "status", st))
                        continue
                    st = lib.mrw_future_wait(fut, 120000)
                    lib.mrw_future_release(fut)
                    out = y.cpu().numpy()
                    got = [OB.digest(inputs.instance_view(out, d)) for d in desc]
                    if st != M.MRW_OK or got != want:
                        errors.append((tid, k, rep, st))
        except Exception as e:  # reported below
            errors.append((tid, repr(e)))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors[:5]
