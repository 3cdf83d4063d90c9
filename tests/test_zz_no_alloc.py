"""The allocation-free batched entry point against the oracle and the regular batched entry point.

mrw_execute_batched_noalloc exists for callers that must not allocate device memory (a framework
whose device memory belongs to its own pool allocator, or a latency-critical loop where
cudaMalloc / cudaFree would synchronise the device): it keeps the stencil kernel's scratch in a
fixed file-scope device array instead. Every instance it writes must equal the oracle's
single-instance evaluation (and the regular batched call's bytes), call after call, although every
call reuses the same array; mrw_noalloc_status must report a tile wait that gave up.
This file is named so that pytest collects it last.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from oracle import image as O
from paper_1510_06585_gb300 import inputs
from paper_1510_06585_gb300 import mrw as M

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _batch(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    shapes = np.stack([rng.integers(1, 400, size=n), rng.integers(1, 300, size=n)], axis=1)
    desc, nbytes = inputs.batch_descriptors(shapes)
    arena = inputs.batch_arena(desc, nbytes, seed=seed)
    return np.ascontiguousarray(desc, dtype=np.int64), arena


def _noalloc(lib, tree, x, y, desc):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.mrw_execute_batched_noalloc(tree.h, x.data_ptr(), y.data_ptr(), x.numel(),
                                           desc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), desc.shape[0],
                                           None, stream)


def _status(lib):
    v = ctypes.c_uint32(77)
    st = lib.mrw_noalloc_status(torch.cuda.current_stream().cuda_stream, ctypes.byref(v))
    return st, v.value


def _check_against_oracle(arena, out, desc, stages):
    for d in desc:  # the trees' noise seed is 0, so each instance's own seed applies
        img = inputs.instance_view(arena, d)
        want = img
        for fn in stages:
            want = fn(want, int(d[4]))
        assert np.array_equal(inputs.instance_view(out, d), want), tuple(d)


FILTER_BLUR = [lambda p, s: O.noise(p, s), lambda p, s: O.solarise(p), lambda p, s: O.mirror(p),
               lambda p, s: O.blur5(p)]


def test_noalloc_matches_oracle_on_two_calls_in_a_row():
    lib = M.load()
    tree = M.map_(M.pipeline(M.stage("noise"), M.stage("solarise"), M.stage("mirror"), M.stage("blur5")))
    for call, (n, seed) in enumerate([(M.MRW_NOALLOC_MAX_INSTANCES, 21), (37, 22)]):
        desc, arena = _batch(n, seed)
        x = torch.from_numpy(arena).cuda()
        got = torch.zeros_like(x)
        st = _noalloc(lib, tree, x, got, desc)
        assert st == M.MRW_OK, lib.mrw_last_error()
        assert _status(lib) == (M.MRW_OK, 0)
        out = got.cpu().numpy()
        _check_against_oracle(arena, out, desc, FILTER_BLUR)
        # and the regular batched call's bytes, padding included
        want = torch.zeros_like(x)
        M.execute_batched(tree, x, want, desc).wait(120000)
        assert torch.equal(got, want), f"call {call}"


@pytest.mark.parametrize("names,stages", [
    # no blur: a pointwise-only tree on the 2-D tile kernel (no halo)
    (["noise", "solarise", "mirror"], [lambda p, s: O.noise(p, s), lambda p, s: O.solarise(p),
                                       lambda p, s: O.mirror(p)]),
    # pointwise stages after the blur (the suffix of the tile kernel), a mirror among them
    (["noise", "blur5", "threshold3", "mirror"], [lambda p, s: O.noise(p, s), lambda p, s: O.blur5(p),
                                                  lambda p, s: O.threshold3(p), lambda p, s: O.mirror(p)]),
])
def test_noalloc_halo_free_and_suffix_trees(names, stages):
    lib = M.load()
    tree = M.map_(M.pipeline(*[M.stage(nm) for nm in names]))
    desc, arena = _batch(53, 24)
    x = torch.from_numpy(arena).cuda()
    got = torch.zeros_like(x)
    assert _noalloc(lib, tree, x, got, desc) == M.MRW_OK, lib.mrw_last_error()
    assert _status(lib) == (M.MRW_OK, 0)
    _check_against_oracle(arena, got.cpu().numpy(), desc, stages)


def test_noalloc_rejects_oversized_batches_multi_kernel_trees_and_capture():
    lib = M.load()
    tree = M.map_(M.pipeline(M.stage("noise"), M.stage("blur5")))
    desc, arena = _batch(M.MRW_NOALLOC_MAX_INSTANCES + 1, 23)
    x = torch.from_numpy(arena).cuda()
    y = torch.zeros_like(x)
    assert _noalloc(lib, tree, x, y, desc) == M.MRW_ERR_INVALID_ARG
    assert b"1 to 256 instances" in lib.mrw_last_error()
    two_blurs = M.map_(M.pipeline(M.stage("blur5"), M.stage("blur5")))
    assert _noalloc(lib, two_blurs, x, y, desc[:4]) == M.MRW_ERR_UNSUPPORTED
    # an instance whose offset is near INT64_MAX lies outside the arena (no overflow in the check)
    far = desc[:2].copy()
    far[1, 0] = (1 << 63) - 16
    assert _noalloc(lib, tree, x, y, far) == M.MRW_ERR_SHAPE
    # inside a stream capture the call refuses and enqueues nothing
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    rc = []
    with torch.cuda.graph(g, stream=side):
        rc.append(_noalloc(lib, tree, x, y, desc[:4]))
        y.add_(0)
    assert rc == [M.MRW_ERR_UNSUPPORTED]
    assert b"captured" in lib.mrw_last_error()
    assert lib.mrw_noalloc_status(None, None) == M.MRW_ERR_INVALID_ARG


def test_noalloc_status_reports_a_wait_that_gave_up():
    # A child process makes every tile wait give up at once (the failure-detection hook): the
    # kernel records the failure in the array's status word and leaves; mrw_noalloc_status reports
    # it, and the next call (hook removed) clears it and writes the oracle's bytes.
    code = r"""
import ctypes, os, sys
import numpy as np, torch
sys.path.insert(0, %r)
from oracle import image as O
from paper_1510_06585_gb300 import mrw as M, inputs
lib = M.load()
shapes = np.array([[70, 40], [130, 9], [300, 200]], dtype=np.int64)
desc, nbytes = inputs.batch_descriptors(shapes)
desc = np.ascontiguousarray(desc, dtype=np.int64)
arena = inputs.batch_arena(desc, nbytes, seed=3)
x = torch.from_numpy(arena).cuda(); y = torch.zeros_like(x)
tree = M.map_(M.pipeline(M.stage("noise"), M.stage("blur5")))
s = torch.cuda.current_stream().cuda_stream
dp = desc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
def run():
    return lib.mrw_execute_batched_noalloc(tree.h, x.data_ptr(), y.data_ptr(), x.numel(), dp, 3, None, s)
v = ctypes.c_uint32(0)
print("call", run())
print("status", lib.mrw_noalloc_status(s, ctypes.byref(v)), v.value)
os.environ.pop("MRW_TEST_WAIT_POLLS")
print("call2", run())
print("status2", lib.mrw_noalloc_status(s, ctypes.byref(v)), v.value)
out = y.cpu().numpy()
ok = all(np.array_equal(inputs.instance_view(out, d), O.blur5(O.noise(inputs.instance_view(arena, d), int(d[4]))))
         for d in desc)
print("oracle", ok)
""" % ROOT
    env = dict(os.environ, MRW_TEST_WAIT_POLLS="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "call 0" in r.stdout and "call2 0" in r.stdout, r.stdout
    assert "status %d 1" % M.MRW_ERR_DEVICE in r.stdout, r.stdout
    assert "status2 0 0" in r.stdout, r.stdout
    assert "oracle True" in r.stdout, r.stdout
