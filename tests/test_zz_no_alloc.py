"""The allocation-free batched entry point against the regular batched entry point.

mrw_execute_batched_noalloc exists for callers that must not allocate device memory (a framework
whose device memory belongs to its own pool allocator, or a latency-critical loop where
cudaMalloc / cudaFree would synchronise the device): it keeps the stencil kernel's scratch in a
fixed file-scope device array instead. Its output must be byte-for-byte the output of
mrw_execute_batched, call after call, although every call reuses the same array.
This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1510_06585_gb300 import inputs
from paper_1510_06585_gb300 import mrw as M

pytestmark = pytest.mark.gpu


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


def test_noalloc_matches_batched_on_two_calls_in_a_row():
    lib = M.load()
    tree = M.map_(M.pipeline(M.stage("noise"), M.stage("solarise"), M.stage("mirror"), M.stage("blur5")))
    for call, (n, seed) in enumerate([(M.MRW_NOALLOC_MAX_INSTANCES, 21), (37, 22)]):
        desc, arena = _batch(n, seed)
        x = torch.from_numpy(arena).cuda()
        want = torch.zeros_like(x)
        M.execute_batched(tree, x, want, desc).wait(120000)
        got = torch.zeros_like(x)
        st = _noalloc(lib, tree, x, got, desc)
        assert st == M.MRW_OK, lib.mrw_last_error()
        torch.cuda.synchronize()
        assert torch.equal(got, want), f"call {call}"


def test_noalloc_rejects_oversized_batches_and_multi_kernel_trees():
    lib = M.load()
    tree = M.map_(M.pipeline(M.stage("noise"), M.stage("blur5")))
    desc, arena = _batch(M.MRW_NOALLOC_MAX_INSTANCES + 1, 23)
    x = torch.from_numpy(arena).cuda()
    y = torch.zeros_like(x)
    assert _noalloc(lib, tree, x, y, desc) == M.MRW_ERR_INVALID_ARG
    assert b"1 to 256 instances" in lib.mrw_last_error()
    two_blurs = M.map_(M.pipeline(M.stage("blur5"), M.stage("blur5")))
    assert _noalloc(lib, two_blurs, x, y, desc[:4]) == M.MRW_ERR_UNSUPPORTED
