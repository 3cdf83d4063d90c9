"""GPU checks of the autotuner, the knowledge base lookup, futures and the bounded-wait error path."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from gpu_util import build_image_tree, empty_like_device, to_device
from oracle import image as O
from paper_1510_06585_gb300 import inputs
from paper_1510_06585_gb300 import mrw as M

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_measure_and_exhaustive_tune_record_the_best():
    M.load().mrw_kb_clear()
    img = inputs.filter_image(1024, 2048)
    x, y = to_device(img), empty_like_device(img)
    tree = build_image_tree(["noise", "solarise", "mirror"], {0: 2})
    cfgs = M.tune_candidates(tree, [x, y])
    t = M.tune_measure(tree, [x, y], cfgs, reps=3)
    assert (t > 0).all()
    best, ms = M.tune(tree, [x, y], M.MRW_TUNE_EXHAUSTIVE, reps=3)
    assert ms > 0 and M.load().mrw_kb_size() == 1
    # the fused configurations beat kernel-per-stage on this tree
    assert t[:8].min() < t[8:].min()
    # execute without a config now uses the recorded one (visible through the plan)
    plan = M.plan_describe(tree, [x, y])
    assert plan["groups"][0]["block"] == min(best.block, 256)
    M.execute(tree, [x, y]).wait(60000)
    assert np.array_equal(y.cpu().numpy(), O.filter_pipeline(img, 2))
    pruned, pms = M.tune(tree, [x, y], M.MRW_TUNE_PRUNED, reps=3)
    assert pms > 0
    M.load().mrw_kb_clear()


def test_model_mode_uses_the_installed_model():
    img = inputs.filter_image(256, 256)
    x, y = to_device(img), empty_like_device(img)
    tree = build_image_tree(["noise", "mirror"], {0: 1})
    cfgs = M.tune_candidates(tree, [x, y])
    m = M.Model(16, 64, seed=3)
    m.install(cfgs)
    try:
        best, ms = M.tune(tree, [x, y], M.MRW_TUNE_MODEL)
        f = M.features(tree, [x, y])
        out = torch.zeros(1, 16, device="cuda")
        m.forward(torch.from_numpy(f[None, :]).cuda(), out)
        torch.cuda.synchronize()
        assert best.as_tuple() == cfgs[int(out.argmin())].as_tuple()
    finally:
        M.load().mrw_tune_set_model(None, None, 0)
        M.load().mrw_kb_clear()


def test_future_timeout_leaves_the_future_valid():
    n = 65536
    xs, vs, as_ = inputs.nbody(n)
    st = [torch.from_numpy(t).cuda() for t in (xs, vs, as_)]
    tree = M.loop(M.stage("nbody_kdk", eps=1e-3, dt=1e-3), 50)
    f = M.execute(tree, st)
    s = M.load().mrw_future_wait(f.h, 0)
    assert s in (M.MRW_OK, M.MRW_ERR_TIMEOUT)
    f.wait(600000)


def test_bounded_wait_gives_up_and_reports_without_hanging():
    # A child process runs a stencil group whose tile wait is told to give up at once; the
    # kernel records the failure in its status word and leaves; the future reports it and the
    # stream stays usable.
    code = r"""
import numpy as np, torch, sys
sys.path.insert(0, %r)
from paper_1510_06585_gb300 import mrw as M, inputs
img = inputs.filter_image(64, 64)
x = torch.from_numpy(img).cuda(); y = torch.zeros_like(x)
f = M.execute(M.pipeline(M.stage("blur5")), [x, y])
s = M.load().mrw_future_wait(f.h, 60000)
print("status", s)
import os
os.environ.pop("MRW_TEST_WAIT_POLLS")
g = M.execute(M.pipeline(M.stage("blur5")), [x, y]); g.wait(60000)
print("after", int(y.sum().item()) > 0)
""" % ROOT
    env = dict(os.environ, MRW_TEST_WAIT_POLLS="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "status %d" % M.MRW_ERR_DEVICE in r.stdout, r.stdout
    assert "after True" in r.stdout, r.stdout
