"""mrw_future_result through the C ABI (Section 2.1: a run returns a future of its result): the
MapReduce class counts of the 512^3 segmentation against the oracle, with and without a result
buffer, on device, pinned and pageable host inputs, on the replayed launch, and its errors."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import image as O
from oracle import skeleton as S
from paper_1510_06585_gb300 import inputs
from paper_1510_06585_gb300 import mrw as M
from gpu_util import empty_like_device, to_device

pytestmark = pytest.mark.gpu


def _run(lib, tree, tensors):
    arr = M.buffers(*tensors)
    fut = ctypes.c_void_p()
    M.check(lib.mrw_execute(tree.h, arr, len(tensors), None, M.stream_handle(), ctypes.byref(fut)), "execute")
    return fut


def _result(lib, fut, n=3):
    out = np.full(n, -5, dtype=np.int64)
    M.check(lib.mrw_future_result(fut, out.ctypes.data, out.nbytes), "mrw_future_result")
    return out


def test_segmentation_512_cubed_counts_come_back_through_the_future():
    lib = M.load()
    vol = inputs.volume(512, 512, 512)
    labels_w, counts_w = O.segmentation(vol)
    x = torch.from_numpy(vol).cuda()
    y = torch.empty_like(x)
    tree = M.mapreduce(M.map_(M.stage("threshold3")))
    # no args[2]: the future owns the result
    fut = _run(lib, tree, [x, y])
    try:
        assert np.array_equal(_result(lib, fut), counts_w)
        assert np.array_equal(_result(lib, fut), counts_w)  # asked twice: the same values
    finally:
        lib.mrw_future_release(fut)
    assert np.array_equal(y.cpu().numpy(), labels_w)
    # with args[2] on the device: the future reads it; the second identical call is replayed
    c = torch.full((3,), -1, dtype=torch.int64, device="cuda")
    for _ in range(2):
        fut = _run(lib, tree, [x, y, c])
        try:
            assert np.array_equal(_result(lib, fut), counts_w)
        finally:
            lib.mrw_future_release(fut)
    assert np.array_equal(c.cpu().numpy(), counts_w)


def test_result_on_host_inputs_and_sum_reduction():
    lib = M.load()
    vol = inputs.volume(40, 512, 520, seed=13)  # > 8 MiB pageable: the chunked staging path
    labels_w, counts_w = O.segmentation(vol)
    out = np.zeros_like(vol)
    tree = M.mapreduce(M.map_(M.stage("threshold3")))
    fut = _run(lib, tree, [vol, out])
    try:
        assert np.array_equal(_result(lib, fut), counts_w)
    finally:
        lib.mrw_future_release(fut)
    assert np.array_equal(out, labels_w)
    pin_in = torch.from_numpy(vol[:8]).pin_memory()  # pinned: read and written in place
    pin_out = torch.zeros_like(pin_in).pin_memory()
    fut = _run(lib, tree, [pin_in, pin_out])
    try:
        assert np.array_equal(_result(lib, fut), O.segmentation(vol[:8])[1])
    finally:
        lib.mrw_future_release(fut)
    # + over a noisy chain: one int64 value
    img = inputs.filter_image(77, 301, seed=3)
    names = [("stage", "noise", {"seed": 5}), ("stage", "solarise", {})]
    want, total = S.evaluate_image(("mapreduce", ("pipeline", names), "add"), img)
    st = M.mapreduce(M.map_(M.pipeline(M.stage("noise", seed=5), M.stage("solarise"))))
    xi, yi = to_device(img), empty_like_device(img)  # rows padded to a 16-byte pitch
    fut = _run(lib, st, [xi, yi])
    try:
        assert _result(lib, fut, 1)[0] == total[0]
    finally:
        lib.mrw_future_release(fut)


def test_result_errors():
    lib = M.load()
    img = inputs.filter_image(16, 32)
    x = torch.from_numpy(img).cuda()
    y = torch.empty_like(x)
    fut = _run(lib, M.pipeline(M.stage("solarise")), [x, y])
    out = np.zeros(3, dtype=np.int64)
    try:  # no reduction in the tree
        assert lib.mrw_future_result(fut, out.ctypes.data, out.nbytes) == M.MRW_ERR_INVALID_ARG
    finally:
        lib.mrw_future_release(fut)
    fut = _run(lib, M.mapreduce(M.map_(M.stage("threshold3"))), [x, y])
    try:  # too small a destination; then the right size
        assert lib.mrw_future_result(fut, out.ctypes.data, 16) == M.MRW_ERR_INVALID_ARG
        assert lib.mrw_future_result(fut, None, 24) == M.MRW_ERR_INVALID_ARG
        assert np.array_equal(_result(lib, fut), O.segmentation(img)[1])
    finally:
        lib.mrw_future_release(fut)
