"""Repeated executions of one tree. A call whose tree, arguments, configuration, stream and device
equal the previous call's (on the same thread) replays the chain launch that call prepared; any
change in between (another buffer, a tree that grew, a knowledge-base or cost-model change,
another stream) makes the executor plan again. Every result against the oracle, bit-exact."""

import numpy as np
import pytest
import torch

from gpu_util import build_image_tree, empty_like_device, oracle_tree, to_device
from oracle import skeleton as S
from paper_1510_06585_gb300 import inputs
from paper_1510_06585_gb300 import mrw as M

pytestmark = pytest.mark.gpu

NAMES = ["noise", "solarise", "mirror"]
SEEDS = {0: 2}


def _run(tree, args, cfg=None, stream=None):
    M.execute(tree, args, cfg, stream=stream).wait(60000)


def test_replayed_calls_give_the_oracle_bytes_every_time():
    img = inputs.filter_image(67, 301, seed=9)
    want, _ = S.evaluate_image(oracle_tree(NAMES, SEEDS), img)
    x, y = to_device(img), empty_like_device(img)
    tree = build_image_tree(NAMES, SEEDS)
    for cfg in (None, M.config(), M.config(block=128, ctas_per_sm=2, unroll=2), M.config(fusion=M.MRW_FUSE_NONE)):
        for _ in range(3):
            y.fill_(0)
            _run(tree, [x, y], cfg)
            assert np.array_equal(y.cpu().numpy(), want), cfg
    # a timed execution of the same call replays too, and still records its time
    f = M.execute(tree, [x, y], None, timed=True)
    f.wait(60000)
    assert f.elapsed_ms() > 0
    assert np.array_equal(y.cpu().numpy(), want)


def test_other_buffers_and_streams_plan_again():
    img = inputs.filter_image(40, 160, seed=3)
    img2 = inputs.filter_image(40, 160, seed=4)
    tree = build_image_tree(NAMES, SEEDS)
    otree = oracle_tree(NAMES, SEEDS)
    x, x2 = to_device(img), to_device(img2)
    y, y2 = empty_like_device(img), empty_like_device(img)
    _run(tree, [x, y])
    _run(tree, [x2, y2])  # same tree, other buffers
    assert np.array_equal(y.cpu().numpy(), S.evaluate_image(otree, img)[0])
    assert np.array_equal(y2.cpu().numpy(), S.evaluate_image(otree, img2)[0])
    # a view of other rows: the same pointer, another shape
    _run(tree, [x[:20], y[:20]])
    _run(tree, [x, y])
    assert np.array_equal(y.cpu().numpy(), S.evaluate_image(otree, img)[0])
    side = torch.cuda.Stream()
    y.fill_(0)
    _run(tree, [x, y], stream=side)
    assert np.array_equal(y.cpu().numpy(), S.evaluate_image(otree, img)[0])


def test_a_tree_that_grows_is_planned_again():
    img = inputs.filter_image(33, 200, seed=5)
    x, y = to_device(img), empty_like_device(img)
    tree = build_image_tree(NAMES, SEEDS)
    _run(tree, [x, y])
    _run(tree, [x, y])
    lib = M.load()
    M.check(lib.mrw_pipeline_add_stage(tree.h, M.STAGE_BY_NAME["threshold3"], None), "add_stage")
    _run(tree, [x, y])
    want, _ = S.evaluate_image(oracle_tree(NAMES + ["threshold3"], SEEDS), img)
    assert np.array_equal(y.cpu().numpy(), want)
    extra = M.stage("solarise")
    M.check(lib.mrw_pipeline_add_node(tree.h, extra.h), "add_node")
    _run(tree, [x, y])
    want, _ = S.evaluate_image(oracle_tree(NAMES + ["threshold3", "solarise"], SEEDS), img)
    assert np.array_equal(y.cpu().numpy(), want)


def test_alternating_trees_and_a_mapreduce():
    vol = inputs.volume(4, 30, 96, seed=6)
    x, y = to_device(vol), empty_like_device(vol)
    red = torch.zeros(3, dtype=torch.int64, device="cuda")
    seg = M.mapreduce(M.map_(M.stage("threshold3")))
    filt = build_image_tree(NAMES, SEEDS)
    want_lab, want_counts = S.evaluate_image(("mapreduce", ("map", ("stage", "threshold3", {})), "add"), vol)
    want_filt, _ = S.evaluate_image(oracle_tree(NAMES, SEEDS), vol)
    for _ in range(3):
        red.fill_(-1)
        _run(seg, [x, y, red])
        assert np.array_equal(y.cpu().numpy(), want_lab) and np.array_equal(red.cpu().numpy(), want_counts)
        _run(filt, [x, y])
        assert np.array_equal(y.cpu().numpy(), want_filt)
    for _ in range(3):  # the same MapReduce call back to back: replayed (chain and finish kernel), counts overwritten
        red.fill_(-1)
        _run(seg, [x, y, red])
        assert np.array_equal(red.cpu().numpy(), want_counts)


def test_a_knowledge_base_change_is_seen():
    img = inputs.filter_image(64, 512, seed=7)
    x, y = to_device(img), empty_like_device(img)
    tree = build_image_tree(NAMES, SEEDS)
    want, _ = S.evaluate_image(oracle_tree(NAMES, SEEDS), img)
    M.check(M.load().mrw_kb_clear(), "kb_clear")
    _run(tree, [x, y])
    _run(tree, [x, y])
    M.tune(tree, [x, y], M.MRW_TUNE_EXHAUSTIVE, reps=1)  # records a configuration for this workload
    y.fill_(0)
    _run(tree, [x, y])
    d = M.plan_describe(tree, [x, y])
    assert len(d["groups"]) == 1 and np.array_equal(y.cpu().numpy(), want)
    M.check(M.load().mrw_kb_clear(), "kb_clear")
    y.fill_(0)
    _run(tree, [x, y])
    assert np.array_equal(y.cpu().numpy(), want)
