"""GPU parity of the fused pointwise chain (Filter Pipeline, Map / MapReduce segmentation) against
the CPU oracle: bit-exact for every integer stage."""
import numpy as np
import pytest
import torch

from gpu_util import build_image_tree, empty_like_device, oracle_tree, round_up, run_image, to_device
from oracle import image as O
from oracle import skeleton as S
from paper_1510_06585_gb300 import inputs
from paper_1510_06585_gb300 import mrw as M

pytestmark = pytest.mark.gpu

FILTER = ["noise", "solarise", "mirror"]


def test_filter_pipeline_1024_fused_and_unfused():
    img = inputs.filter_image(1024, 1024)
    want = O.filter_pipeline(img, inputs.SEED_NOISE)
    tree = build_image_tree(FILTER, {0: inputs.SEED_NOISE})
    for cfg in (None, M.config(), M.config(fusion=M.MRW_FUSE_NONE)):
        got, _ = run_image(tree, img, cfg)
        assert np.array_equal(got, want)


def test_filter_pipeline_8192_every_candidate_config():
    # the roofline-sweep size: every launch shape the tuner may pick (unroll 1..8, persistent and
    # blocked row orders, prefetching of the next rows) gives the oracle's bytes on 67 M pixels
    img = inputs.filter_image(8192, 8192)
    want = O.filter_pipeline(img, inputs.SEED_NOISE)
    tree = build_image_tree(FILTER, {0: inputs.SEED_NOISE})
    x, y = to_device(img), empty_like_device(img)
    cfgs = M.tune_candidates(tree, [x, y])
    assert len(cfgs) == 16
    for c in cfgs:
        y.zero_()
        M.execute(tree, [x, y], c).wait(60000)
        assert np.array_equal(y.cpu().numpy(), want), c.as_tuple()


def test_filter_pipeline_odd_widths_and_8x8_brute_force():
    tree = build_image_tree(FILTER, {0: 2})
    for (h, w) in [(8, 8), (1, 1), (3, 7)] + [(5, k) for k in range(1, 34)] + [(7, 1000), (2, 1023), (3, 4097)]:
        img = inputs.filter_image(h, w, seed=1000 + w)
        got, _ = run_image(tree, img)
        assert np.array_equal(got, O.filter_pipeline(img, 2)), (h, w)


def test_padded_pitches():
    tree = build_image_tree(FILTER, {0: 9})
    for (h, w, pitch) in [(9, 17, 48), (4, 100, 256), (6, 16, 16), (3, 31, 4096)]:
        img = inputs.filter_image(h, w, seed=w)
        got, _ = run_image(tree, img, pitch=pitch)
        assert np.array_equal(got, O.filter_pipeline(img, 9)), (h, w, pitch)


def test_output_padding_bytes_are_not_written():
    img = inputs.filter_image(10, 21)
    x = to_device(img, 64)
    y = empty_like_device(img, 64, fill=0xAB)
    M.execute(build_image_tree(FILTER, {0: 2}), [x, y]).wait(60000)
    store = y.as_strided((10, 64), (64, 1)).cpu().numpy()
    assert (store[:, 21:] == 0xAB).all()


@pytest.mark.parametrize("seed", range(12))
def test_random_chains_match_depth_first_oracle(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    names = [("noise", "solarise", "mirror", "threshold3")[int(k)] for k in rng.integers(0, 4, size=int(rng.integers(1, 9)))]
    seeds = {i: int(rng.integers(0, 2 ** 32)) for i in range(len(names))}
    h, w = int(rng.integers(1, 40)), int(rng.integers(1, 300))
    img = inputs.filter_image(h, w, seed=seed)
    want, _ = S.evaluate_image(oracle_tree(names, seeds), img)
    tree = build_image_tree(names, seeds)
    for cfg in (M.config(), M.config(fusion=M.MRW_FUSE_NONE), M.config(block=128, ctas_per_sm=2, unroll=1)):
        got, _ = run_image(tree, img, cfg)
        assert np.array_equal(got, want), (names, h, w)


@pytest.mark.parametrize("names", [
    ["noise"], ["solarise"], ["threshold3"], ["noise", "solarise"], ["mirror", "noise", "mirror", "solarise"],
    ["solarise", "noise"], ["noise", "solarise", "mirror", "solarise"], ["threshold3", "solarise"], ["mirror"],
])
def test_op_sequences_with_and_without_fast_paths(names):
    # the kernels run the common sequences (one noise, one solarise, one threshold, noise then
    # solarise; mirrors do not count) without walking the op list; near misses take the general path
    seeds = {i: 40 + i for i in range(len(names))}
    tree = build_image_tree(names, seeds)
    for (h, w) in [(37, 301), (64, 1024), (5, 17)]:
        img = inputs.filter_image(h, w, seed=h * w)
        want, _ = S.evaluate_image(oracle_tree(names, seeds), img)
        for cfg in (M.config(), M.config(unroll=1), M.config(unroll=4), M.config(unroll=8)):
            got, _ = run_image(tree, img, cfg)
            assert np.array_equal(got, want), (names, h, w, cfg.as_tuple())


def test_every_candidate_config_gives_the_same_bytes():
    img = inputs.filter_image(333, 517, seed=5)
    tree = build_image_tree(["noise", "mirror", "solarise", "noise"], {0: 3, 3: 4})
    want, _ = S.evaluate_image(oracle_tree(["noise", "mirror", "solarise", "noise"], {0: 3, 3: 4}), img)
    for c in M.tune_candidates(tree, [img, img]):
        got, _ = run_image(tree, img, c)
        assert np.array_equal(got, want), c.as_tuple()


def test_volume_rows_are_counted_across_planes():
    vol = inputs.volume(3, 5, 40, seed=2)
    tree = M.map_(build_image_tree(["noise", "mirror"], {0: 77}))
    got, _ = run_image(tree, vol)
    assert np.array_equal(got, O.mirror(O.noise(vol, 77)))


def test_segmentation_small_volumes():
    for (d, h, w) in [(1, 1, 1), (2, 3, 17), (8, 64, 100), (4, 33, 512)]:
        vol = inputs.volume(d, h, w, seed=d * w)
        tree = M.mapreduce(M.map_(M.stage("threshold3")))
        labels_w, counts_w = O.segmentation(vol)
        for cfg in (M.config(), M.config(fusion=M.MRW_FUSE_NONE)):
            labels, counts = run_image(tree, vol, cfg, reduce_k=3)
            assert np.array_equal(labels, labels_w) and np.array_equal(counts, counts_w), (d, h, w)


def test_segmentation_512_cubed_full_size():
    vol = inputs.volume(512, 512, 512)
    tree = M.mapreduce(M.map_(M.stage("threshold3")))
    labels, counts = run_image(tree, vol, None, reduce_k=3)
    hist, _ = np.histogram(vol, bins=[0, 85, 170, 256])
    assert np.array_equal(counts, hist.astype(np.int64))
    assert counts.sum() == 512 ** 3
    # labels: compare plane chunks against the oracle stage
    for z in range(0, 512, 64):
        assert np.array_equal(labels[z:z + 64], O.threshold3(vol[z:z + 64])), z


def test_mapreduce_sum_of_a_noisy_chain():
    img = inputs.filter_image(77, 301, seed=3)
    names = ["noise", "solarise"]
    tree = M.mapreduce(M.map_(build_image_tree(names, {0: 5})))
    out, red = run_image(tree, img, reduce_k=1)
    want, total = S.evaluate_image(("mapreduce", oracle_tree(names, {0: 5}), "add"), img)
    assert np.array_equal(out, want) and red[0] == total[0]


def test_loop_of_a_chain():
    img = inputs.filter_image(19, 45, seed=4)
    body = build_image_tree(FILTER, {0: 8})
    got, _ = run_image(M.loop(body, 3), img)
    want, _ = S.evaluate_image(("loop", oracle_tree(FILTER, {0: 8}), 3), img)
    assert np.array_equal(got, want)


def test_host_buffers_are_staged():
    img = inputs.filter_image(200, 301, seed=6)
    out = np.zeros_like(img)
    tree = build_image_tree(FILTER, {0: 2})
    M.execute(tree, [img, out]).wait(60000)
    assert np.array_equal(out, O.filter_pipeline(img, 2))
    pinned_in = torch.from_numpy(img).pin_memory()
    pinned_out = torch.zeros_like(pinned_in).pin_memory()
    counts = torch.zeros(3, dtype=torch.int64).pin_memory()
    seg = M.mapreduce(M.map_(M.stage("threshold3")))
    M.execute(seg, [pinned_in, pinned_out, counts]).wait(60000)
    labels_w, counts_w = O.segmentation(img)
    assert np.array_equal(pinned_out.numpy(), labels_w) and np.array_equal(counts.numpy(), counts_w)


def test_in_place_pointwise_chain():
    img = inputs.filter_image(64, 256, seed=7)
    x = to_device(img)
    M.execute(build_image_tree(["noise", "solarise"], {0: 1}), [x, x]).wait(60000)
    assert np.array_equal(x.cpu().numpy(), O.solarise(O.noise(img, 1)))
    with pytest.raises(M.MrwError):
        M.execute(build_image_tree(FILTER, {0: 1}), [x, x])


def test_future_elapsed_and_query():
    img = inputs.filter_image(512, 512)
    x, y = to_device(img), empty_like_device(img)
    tree = build_image_tree(FILTER, {0: 2})
    f = M.execute(tree, [x, y], timed=True)
    f.wait(60000)
    assert f.elapsed_ms() > 0
    assert M.load().mrw_future_query(f.h) == M.MRW_OK
    assert np.array_equal(y.cpu().numpy(), O.filter_pipeline(img, 2))
    # an untimed future (the default) has no device time to report
    g = M.execute(tree, [x, y])
    g.wait(60000)
    with pytest.raises(M.MrwError) as e:
        g.elapsed_ms()
    assert e.value.status == M.MRW_ERR_INVALID_ARG


def test_pinned_host_buffers_are_read_and_written_in_place():
    # page-locked host buffers with 16-byte rows: the single fused kernel reads and writes them in
    # place over the host link; counts, the noise hash's global rows and a pageable output (staged
    # path) must all give the oracle's bytes
    vol = inputs.volume(24, 256, 512, seed=21)
    pin_in = torch.from_numpy(vol).pin_memory()
    pin_out = torch.zeros_like(pin_in).pin_memory()
    counts = torch.full((3,), -1, dtype=torch.int64).pin_memory()
    seg = M.mapreduce(M.map_(M.stage("threshold3")))
    for _ in range(2):
        M.execute(seg, [pin_in, pin_out, counts]).wait(120000)
        labels_w, counts_w = O.segmentation(vol)
        assert np.array_equal(pin_out.numpy(), labels_w) and np.array_equal(counts.numpy(), counts_w)
    img = inputs.filter_image(1024, 2048, seed=3)
    pi = torch.from_numpy(img).pin_memory()
    po = torch.zeros_like(pi).pin_memory()
    M.execute(build_image_tree(FILTER, {0: 2}), [pi, po]).wait(120000)
    assert np.array_equal(po.numpy(), O.filter_pipeline(img, 2))
    pageable = np.zeros_like(img)
    M.execute(build_image_tree(FILTER, {0: 2}), [pi, pageable]).wait(120000)
    assert np.array_equal(pageable, O.filter_pipeline(img, 2))


def test_large_host_buffers_take_the_overlapped_chunked_path():
    # above 8 MiB the host rows are staged in chunks whose copies overlap the kernels; each chunk's
    # noise hash uses its global row (Offset trait) and the counts accumulate across chunks
    img = inputs.filter_image(3000, 3001, seed=12)
    out = np.zeros_like(img)
    M.execute(build_image_tree(FILTER, {0: 2}), [img, out]).wait(120000)
    assert np.array_equal(out, O.filter_pipeline(img, 2))
    vol = inputs.volume(40, 512, 520, seed=13)
    pin_in = torch.from_numpy(vol).pin_memory()
    pin_out = torch.zeros_like(pin_in).pin_memory()
    counts = torch.full((3,), -1, dtype=torch.int64).pin_memory()
    seg = M.mapreduce(M.map_(M.stage("threshold3")))
    for _ in range(2):  # a second call reuses pooled events and streams
        M.execute(seg, [pin_in, pin_out, counts]).wait(120000)
        labels_w, counts_w = O.segmentation(vol)
        assert np.array_equal(pin_out.numpy(), labels_w) and np.array_equal(counts.numpy(), counts_w)
