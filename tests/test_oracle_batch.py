"""Pins of oracle.batch (no GPU): the per-instance digests equal the digests of the instances
evaluated in full by the depth-first oracle on the arena the executor is given, in one process
and in a spawned pool."""
import numpy as np

from oracle import batch as B
from oracle import skeleton as S
from paper_1510_06585_gb300 import inputs


def _tree(seed):
    names = ["noise", "solarise", "mirror", "blur5"]
    return ("pipeline", [("stage", n, {"seed": seed if n == "noise" else 0}) for n in names])


def test_digests_match_full_evaluation_of_the_arena():
    shapes = inputs.batch_shapes(12, lo=8, hi=90)
    desc, nbytes = inputs.batch_descriptors(shapes)
    arena = inputs.batch_arena(desc, nbytes)
    want = []
    for i in range(len(desc)):
        out, _ = S.evaluate_image(_tree(int(desc[i, 4])), inputs.instance_view(arena, desc[i]))
        want.append(B.digest(out))
    assert B.batch_digests(desc, processes=1) == want
    assert B.batch_digests(desc, processes=2) == want
    # a changed pixel changes its instance's digest only
    out0, _ = S.evaluate_image(_tree(int(desc[0, 4])), inputs.instance_view(arena, desc[0]))
    out0 = out0.copy()
    out0[0, 0] ^= 1
    assert B.digest(out0) != want[0]


def test_instance_generator_is_the_arena_content():
    shapes = np.array([[17, 5], [40, 33]])
    desc, nbytes = inputs.batch_descriptors(shapes)
    arena = inputs.batch_arena(desc, nbytes)
    for i in range(2):
        w, h = int(desc[i, 1]), int(desc[i, 2])
        assert np.array_equal(inputs.instance_view(arena, desc[i]), inputs.batch_instance(i, w, h))
