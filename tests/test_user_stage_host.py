"""User-defined stages (mrw_stage_user) on the host, no GPU: argument checks, the run-time
compiler's error reporting, and the oracle's user leaf against a direct numpy composition."""
import numpy as np
import pytest

from oracle import image as O
from oracle import skeleton as S
from paper_1510_06585_gb300 import inputs
from paper_1510_06585_gb300 import mrw as M

INVERT = "__device__ unsigned char invert(unsigned char p, int x, int y, const unsigned int *u) {\n" \
         "  return (unsigned char)(255 - p);\n}\n"


def _build_or_skip(name, src, params=None):
    try:
        return M.user_stage(name, src, params)
    except M.MrwError as e:
        if "NVRTC" in str(e) and "not found" in str(e):
            pytest.skip("NVRTC is not installed")
        raise


def test_user_stage_builds_and_rejects_bad_arguments():
    node = _build_or_skip("invert", INVERT)
    assert node.h
    for name, src in [("", INVERT), ("invert", ""), ("1invert", INVERT), ("in-vert", INVERT), ("x" * 64, INVERT)]:
        with pytest.raises(M.MrwError) as e:
            M.user_stage(name, src)
        assert e.value.status == M.MRW_ERR_INVALID_ARG, (name, src[:10])
    with pytest.raises(ValueError):
        M.user_stage("invert", INVERT, list(range(9)))


def test_user_stage_compile_errors_carry_the_compiler_log():
    _build_or_skip("invert", INVERT)
    bad = "__device__ unsigned char f(unsigned char p, int x, int y, const unsigned int *u) { return undefined_q; }"
    with pytest.raises(M.MrwError) as e:
        M.user_stage("f", bad)
    assert e.value.status == M.MRW_ERR_UNSUPPORTED
    assert "undefined_q" in str(e.value) and "error" in str(e.value)
    # the named function must exist with the documented signature
    with pytest.raises(M.MrwError) as e:
        M.user_stage("g", INVERT)
    assert e.value.status == M.MRW_ERR_UNSUPPORTED
    with pytest.raises(M.MrwError) as e:
        M.user_stage("invert", INVERT.replace("const unsigned int *u", "float u"))
    assert e.value.status == M.MRW_ERR_UNSUPPORTED


def test_user_stages_join_pipelines_and_loops_on_the_host():
    node = _build_or_skip("invert", INVERT)
    tree = M.pipeline(M.stage("noise", seed=3), node, M.stage("mirror"))
    M.loop(tree, 3)
    M.mapreduce(M.map_(M.pipeline(node, M.stage("threshold3"))))


def test_oracle_user_leaf_is_the_plain_composition():
    img = inputs.filter_image(13, 37, seed=4)

    def ramp(a, y0):  # p * 3 + x + 2 y + 5 (mod 256), x and y global
        h, w = a.shape
        x = np.arange(w, dtype=np.int64)[None, :]
        y = (y0 + np.arange(h, dtype=np.int64))[:, None]
        return ((a.astype(np.int64) * 3 + x + 2 * y + 5) & 0xFF).astype(np.uint8)

    tree = ("pipeline", [("stage", "noise", {"seed": 9}), ("user", ramp), ("stage", "mirror", {}),
                         ("user", lambda a, y0: 255 - a)])
    trace = []
    got, _ = S.evaluate_image(tree, img, trace)
    want = 255 - O.mirror(ramp(O.noise(img, 9), 0))
    assert np.array_equal(got, want) and trace == ["noise", "user", "mirror", "user"]
    # Map over a volume: every plane's rows are global rows (plane k starts at row k H)
    vol = inputs.volume(3, 5, 21, seed=8)
    got, _ = S.evaluate_image(("map", ("user", ramp)), vol)
    assert np.array_equal(got, ramp(vol.reshape(15, 21), 0).reshape(3, 5, 21))
    # and the user leaf is a valid MapReduce terminal (value sum)
    _, total = S.evaluate_image(("mapreduce", ("user", ramp), "add"), img)
    assert total[0] == int(ramp(img, 0).astype(np.int64).sum())
