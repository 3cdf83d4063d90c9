"""GPU parity of user-defined stages (mrw_stage_user): per-pixel CUDA C functions compiled at run
time and fused with the built-in pointwise stages, against the oracle's depth-first walk in which
each user function is its plain numpy definition. Bit-exact."""

import numpy as np
import pytest
import torch

from gpu_util import run_image, to_device, empty_like_device
from oracle import skeleton as S
from paper_1510_06585_gb300 import inputs
from paper_1510_06585_gb300 import mrw as M

pytestmark = pytest.mark.gpu

INVERT_SRC = """__device__ unsigned char invert(unsigned char p, int x, int y, const unsigned int *u) {
  return (unsigned char)(255 - p);
}"""

# p * u0 + x * u1 + y * u2 + u3 (mod 256), x and y the global column and row of the stage's input
RAMP_SRC = """__device__ unsigned int mix(unsigned int a, unsigned int b) { return a * b; }
__device__ unsigned char ramp(unsigned char p, int x, int y, const unsigned int *u) {
  return (unsigned char)((mix(p, u[0]) + mix((unsigned int)x, u[1]) + mix((unsigned int)y, u[2]) + u[3]) & 0xFFu);
}"""


def invert_np(a, y0):
    return (255 - a).astype(np.uint8)


def ramp_np(u):
    def f(a, y0):
        h, w = a.shape
        x = np.arange(w, dtype=np.uint64)[None, :]
        y = (y0 + np.arange(h, dtype=np.uint64))[:, None]
        return ((a.astype(np.uint64) * u[0] + x * u[1] + y * u[2] + u[3]) & 0xFF).astype(np.uint8)
    return f


def build(spec):
    """spec: list of ("noise", seed) / ("solarise",) / ("mirror",) / ("threshold3",) / ("blur5",) /
    ("invert",) / ("ramp", u) -> (device tree, oracle tree)."""
    nodes, leaves = [], []
    for item in spec:
        name = item[0]
        if name == "invert":
            nodes.append(M.user_stage("invert", INVERT_SRC))
            leaves.append(("user", invert_np))
        elif name == "ramp":
            nodes.append(M.user_stage("ramp", RAMP_SRC, item[1]))
            leaves.append(("user", ramp_np(item[1])))
        elif name == "noise":
            nodes.append(M.stage("noise", seed=item[1]))
            leaves.append(("stage", "noise", {"seed": item[1]}))
        else:
            nodes.append(M.stage(name))
            leaves.append(("stage", name, {}))
    return M.pipeline(*nodes), ("pipeline", leaves)


SHAPES = [(1, 1), (3, 17), (37, 301), (64, 1024), (9, 4096 + 5)]


def test_user_stage_alone():
    tree, otree = build([("invert",)])
    for (h, w) in SHAPES:
        img = inputs.filter_image(h, w, seed=h + w)
        got, _ = run_image(tree, img)
        assert np.array_equal(got, 255 - img), (h, w)


@pytest.mark.parametrize("spec", [
    [("noise", 2), ("ramp", (3, 1, 2, 5)), ("mirror",), ("solarise",)],
    [("mirror",), ("ramp", (1, 7, 0, 0)), ("invert",)],
    [("ramp", (5, 0, 3, 11)), ("mirror",), ("noise", 7), ("mirror",), ("ramp", (1, 1, 1, 1)), ("threshold3",)],
    [("invert",), ("invert",), ("noise", 1), ("noise", 2), ("noise", 3)],
])
def test_user_stages_fused_with_builtins(spec):
    tree, otree = build(spec)
    for (h, w) in SHAPES:
        img = inputs.filter_image(h, w, seed=3 * h + w)
        want, _ = S.evaluate_image(otree, img)
        for cfg in (M.config(), M.config(fusion=M.MRW_FUSE_NONE), M.config(block=128, ctas_per_sm=2)):
            got, _ = run_image(tree, img, cfg)
            assert np.array_equal(got, want), (spec, h, w, cfg.as_tuple())
        got, _ = run_image(tree, img, pitch=((w + 15) // 16) * 16 + 32)  # a wider row pitch
        assert np.array_equal(got, want), (spec, h, w, "pitch")


def test_fused_plan_is_one_generated_kernel_and_blurs_split_it():
    tree, _ = build([("noise", 2), ("ramp", (3, 1, 2, 5)), ("mirror",), ("solarise",)])
    img = np.zeros((64, 256), np.uint8)
    x, y = to_device(img), empty_like_device(img)
    plan = M.plan_describe(tree, [x, y])
    assert [g["kernel"] for g in plan["groups"]] == ["user_chain"]
    assert plan["groups"][0]["ops"] == ["noise", "user:ramp", "mirror", "solarise"]
    tree2, _ = build([("invert",), ("blur5",), ("solarise",), ("ramp", (1, 0, 0, 0))])
    plan2 = M.plan_describe(tree2, [x, y])
    assert [g["kernel"] for g in plan2["groups"]][0] == "user_chain"
    assert [g["kernel"] for g in plan2["groups"]][-1] == "user_chain"
    assert len(plan2["groups"]) == 3


@pytest.mark.parametrize("spec", [
    [("invert",), ("blur5",)],
    [("blur5",), ("ramp", (1, 3, 1, 0)), ("threshold3",)],
    [("noise", 4), ("invert",), ("mirror",), ("blur5",), ("solarise",), ("ramp", (2, 0, 0, 1))],
])
def test_user_stages_around_a_blur(spec):
    tree, otree = build(spec)
    for (h, w) in [(5, 7), (129, 250), (64, 1024)]:
        img = inputs.filter_image(h, w, seed=h * w)
        want, _ = S.evaluate_image(otree, img)
        got, _ = run_image(tree, img)
        assert np.array_equal(got, want), (spec, h, w)


def test_map_over_a_volume_counts_rows_across_planes():
    tree, otree = build([("ramp", (1, 0, 1, 0)), ("noise", 5)])
    vol = inputs.volume(4, 33, 100, seed=12)
    want, _ = S.evaluate_image(("map", otree), vol)
    got, _ = run_image(M.map_(tree), vol)
    assert np.array_equal(got, want)


def test_mapreduce_over_user_stages():
    tree, otree = build([("ramp", (1, 2, 0, 0)), ("threshold3",)])
    vol = inputs.volume(6, 40, 120, seed=1)
    want, counts = S.evaluate_image(("mapreduce", otree, "add"), vol)
    got, red = run_image(M.mapreduce(M.map_(tree)), vol, reduce_k=3)
    assert np.array_equal(got, want) and np.array_equal(red, counts)
    tree_s, otree_s = build([("noise", 3), ("invert",)])
    img = inputs.filter_image(77, 301, seed=2)
    want, total = S.evaluate_image(("mapreduce", otree_s, "add"), img)
    got, red = run_image(M.mapreduce(M.map_(tree_s)), img, reduce_k=1)
    assert np.array_equal(got, want) and red[0] == total[0]


def test_loop_and_host_buffers():
    body, obody = build([("invert",), ("noise", 8), ("ramp", (3, 0, 0, 1))])
    img = inputs.filter_image(50, 333, seed=5)
    want, _ = S.evaluate_image(("loop", obody, 3), img)
    got, _ = run_image(M.loop(body, 3), img)
    assert np.array_equal(got, want)
    out = np.zeros_like(img)
    M.execute(M.loop(body, 3), [img, out]).wait(60000)  # pageable host buffers, staged
    assert np.array_equal(out, want)
    pin_in = torch.from_numpy(img).pin_memory()
    pin_out = torch.zeros_like(pin_in).pin_memory()
    M.execute(body, [pin_in, pin_out]).wait(60000)
    want1, _ = S.evaluate_image(obody, img)
    assert np.array_equal(pin_out.numpy(), want1)


def test_user_stages_are_rejected_where_unsupported():
    tree, _ = build([("invert",), ("blur5",)])
    shapes = inputs.batch_shapes(4)
    desc, nbytes = inputs.batch_descriptors(shapes)
    arena = inputs.batch_arena(desc, nbytes)
    x = torch.from_numpy(arena).cuda()
    y = torch.zeros_like(x)
    with pytest.raises(M.MrwError) as e:
        M.execute_batched(M.map_(tree), x, y, desc)
    assert e.value.status == M.MRW_ERR_UNSUPPORTED
    img = inputs.filter_image(16, 64)
    body, _ = build([("invert",), ("blur5",)])
    with pytest.raises(M.MrwError) as e:
        run_image(M.loop(body, 5, M.MRW_LOOP_WHILE_CHANGED), img)
    assert e.value.status == M.MRW_ERR_UNSUPPORTED
