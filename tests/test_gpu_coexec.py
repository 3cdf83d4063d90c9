"""CPU + GPU co-execution (Section 3.3 of the paper: the GPU and the host cores share the rows of a
tree over host buffers, and the balancer moves rows between them): every co-executed run is
bit-exact against the oracle, whatever the split, and the balancer's profile construction settles
on a split whose two times agree."""
import numpy as np
import pytest
import torch

from oracle import image as O
from oracle import skeleton as S
from paper_1510_06585_gb300 import inputs
from paper_1510_06585_gb300 import mrw as M

pytestmark = pytest.mark.gpu


def test_segmentation_512_cubed_co_executed_is_bit_exact_on_every_split():
    vol = inputs.volume(512, 512, 512)
    labels_w = np.empty_like(vol)
    counts_w = np.zeros(3, np.int64)
    for z in range(0, 512, 64):
        labels_w[z:z + 64], c = O.segmentation(vol[z:z + 64])
        counts_w += c
    pin_in = torch.from_numpy(vol).pin_memory()
    pin_out = torch.zeros_like(pin_in).pin_memory()
    counts = torch.full((3,), -1, dtype=torch.int64).pin_memory()
    seg = M.mapreduce(M.map_(M.stage("threshold3")))
    M.Balancer(gpu_share=0.5).execute(seg, [pin_in, pin_out, counts])  # first-touch costs
    bal = M.Balancer(precision=1.0 / 32, search_reps=2)
    trace = []
    for _ in range(12):
        pin_out.zero_()
        r = bal.execute(seg, [pin_in, pin_out, counts])
        trace.append(r)
        assert np.array_equal(counts.numpy(), counts_w), r
        assert torch.equal(pin_out, torch.from_numpy(labels_w)), r
        assert r["gpu_rows"] + r["cpu_rows"] == 512 * 512
    print([(round(t["gpu_share"], 4), round(t["gpu_ms"], 2), round(t["cpu_ms"], 2), round(t["dev"], 3)) for t in trace])
    assert trace[-1]["phase"] == M.MRW_BAL_MONITOR
    # the search ends with both sides busy and their times within a factor 2 of each other
    last = trace[-1]
    assert 0 < last["gpu_rows"] and 0 < last["cpu_rows"]


@pytest.mark.parametrize("share", [0.0, 0.3, 1.0])
def test_filter_pipeline_at_a_fixed_split(share):
    img = inputs.filter_image(1000, 2048, seed=4)
    want = O.filter_pipeline(img, 2)
    tree = M.pipeline(M.stage("noise", seed=2), M.stage("solarise"), M.stage("mirror"))
    pi = torch.from_numpy(img).pin_memory()
    po = torch.zeros_like(pi).pin_memory()
    r = M.Balancer(gpu_share=share).execute(tree, [pi, po])
    assert r["gpu_rows"] == round(share * 1000)
    assert np.array_equal(po.numpy(), want)
    # pageable buffers: the GPU stages its rows through device memory
    out = np.zeros_like(img)
    M.Balancer(gpu_share=share).execute(tree, [img, out])
    assert np.array_equal(out, want)


def test_sum_reduction_into_a_device_result_and_rejections():
    vol = inputs.volume(6, 128, 200, seed=8)
    names = [("stage", "noise", {"seed": 7}), ("stage", "mirror", {}), ("stage", "noise", {"seed": 9}),
             ("stage", "solarise", {})]
    want, total = S.evaluate_image(("mapreduce", ("map", ("pipeline", names)), "add"), vol)
    tree = M.mapreduce(M.map_(M.pipeline(M.stage("noise", seed=7), M.stage("mirror"), M.stage("noise", seed=9),
                                         M.stage("solarise"))))
    out = np.zeros_like(vol)
    s = torch.zeros(1, dtype=torch.int64, device="cuda")
    M.Balancer(gpu_share=0.45).execute(tree, [vol, out, s])
    assert np.array_equal(out, want) and int(s.item()) == int(total[0])
    # device image buffers and trees that do not fuse into one pointwise kernel are refused
    x = torch.from_numpy(vol).cuda()
    with pytest.raises(M.MrwError) as e:
        M.Balancer().execute(M.pipeline(M.stage("solarise")), [x, torch.empty_like(x)])
    assert e.value.status == M.MRW_ERR_UNSUPPORTED
    with pytest.raises(M.MrwError) as e:
        M.Balancer().execute(M.pipeline(M.stage("solarise"), M.stage("blur5")), [vol, out])
    assert e.value.status == M.MRW_ERR_UNSUPPORTED


def test_random_trees_and_splits_match_the_oracle():
    # random pointwise chains (noise seeds, mirrors, solarise, thresholds), with or without a
    # MapReduce root, on images and volumes of odd widths, at random GPU shares: the host workers'
    # rows and the GPU's rows together must be the oracle's output, whatever the split
    rng = np.random.Generator(np.random.PCG64(31))
    kinds = ["noise", "solarise", "mirror", "threshold3"]
    for case in range(12):
        n = int(rng.integers(1, 6))
        names = [kinds[int(k)] for k in rng.integers(0, 4, size=n)]
        while names.count("noise") > 2:  # at most two noise stages fuse into one kernel
            names.remove("noise")
        seeds = {i: int(rng.integers(0, 2 ** 31)) for i, nm in enumerate(names) if nm == "noise"}
        h, w = int(rng.integers(1, 90)), int(rng.integers(1, 300))
        img = (inputs.volume(int(rng.integers(1, 4)), h, w, seed=case) if case % 2 else
               inputs.filter_image(h, w, seed=case))
        body = M.pipeline(*[M.stage(nm, seed=seeds.get(i, 0)) if nm == "noise" else M.stage(nm)
                            for i, nm in enumerate(names)])
        oracle = ("pipeline", [("stage", nm, {"seed": seeds.get(i, 0)}) for i, nm in enumerate(names)])
        reduce = bool(case % 3 == 0)
        share = float(rng.uniform(0, 1))
        out = np.zeros_like(img)
        if reduce:
            tree = M.mapreduce(M.map_(body))
            want, total = S.evaluate_image(("mapreduce", ("map", oracle), "add"), img)
            k = 3 if names[-1] == "threshold3" else 1
            res = np.full(k, -1, np.int64)
            M.Balancer(gpu_share=share).execute(tree, [img, out, res])
            assert np.array_equal(res, total), (case, names, share)
        else:
            tree = M.map_(body)
            want, _ = S.evaluate_image(("map", oracle), img)
            M.Balancer(gpu_share=share).execute(tree, [img, out])
        assert np.array_equal(out, want), (case, names, share, img.shape)
