"""GPU parity of the Saxpy Map (Section 4, Saxpy) against the FP64 oracle (oracle.saxpy): a Map
of k stages fused into one pass, bit-identical to k kernel-per-stage launches, every launch shape,
ragged lengths and host buffers."""
import numpy as np
import pytest
import torch

from oracle import saxpy as S
from paper_1510_06585_gb300 import mrw as M

pytestmark = pytest.mark.gpu


def _vecs(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.normal(size=n).astype(np.float32), rng.normal(size=n).astype(np.float32)


def _tree(alphas):
    return M.map_(M.pipeline(*[M.stage("saxpy", alpha=a) for a in alphas]))


def _run(tree, x, y, cfg=None):
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    M.execute(tree, [xd, yd], cfg).wait(120000)
    return yd.cpu().numpy()


@pytest.mark.parametrize("n", [1, 3, 4, 5, 1023, 1024, 1025, 1_000_003, (1 << 22) + 7])
def test_one_stage_within_the_rounding_bound(n):
    x, y = _vecs(n, n)
    got = _run(_tree([2.5]), x, y)
    err = np.abs(got.astype(np.float64) - S.saxpy_stages(x, y, [2.5]))
    assert (err <= S.error_bound(x, y, [2.5])).all()


def test_fused_stages_equal_kernel_per_stage_bits_and_the_oracle():
    n = 3_000_017
    x, y = _vecs(n, 11)
    alphas = [1.5, -0.25, 3.0, 0.125, -2.0]
    fused = _run(_tree(alphas), x, y)
    unfused = _run(_tree(alphas), x, y, M.config(fusion=M.MRW_FUSE_NONE))
    assert np.array_equal(fused, unfused)  # one fmaf per stage and element, in stage order
    err = np.abs(fused.astype(np.float64) - S.saxpy_stages(x, y, alphas))
    assert (err <= S.error_bound(x, y, alphas)).all()
    for unroll in (1, 2, 8):
        assert np.array_equal(_run(_tree(alphas), x, y, M.config(unroll=unroll)), fused), unroll


def test_a_loop_of_more_stages_than_one_pass_holds():
    n = 100_003
    x, y = _vecs(n, 12)
    tree = M.loop(M.stage("saxpy", alpha=0.5), 100)  # 64 stages in the first pass, 36 in the second
    fused = _run(tree, x, y)
    assert np.array_equal(fused, _run(tree, x, y, M.config(fusion=M.MRW_FUSE_NONE)))
    err = np.abs(fused.astype(np.float64) - S.saxpy_stages(x, y, [0.5] * 100))
    assert (err <= S.error_bound(x, y, [0.5] * 100)).all()


def test_host_vectors_are_staged_and_misaligned_device_vectors_refused():
    n = 10_001
    x, y = _vecs(n, 13)
    y_host = y.copy()
    M.execute(_tree([-1.75]), [x, y_host]).wait(60000)
    assert (np.abs(y_host.astype(np.float64) - S.saxpy_stages(x, y, [-1.75])) <= S.error_bound(x, y, [-1.75])).all()
    xd = torch.from_numpy(np.concatenate([x, x[:1]])).cuda()
    yd = torch.from_numpy(np.concatenate([y, y[:1]])).cuda()
    with pytest.raises(M.MrwError) as e:
        M.execute(_tree([1.0]), [xd[1:], yd[1:]])
    assert e.value.status == M.MRW_ERR_CONSTRAINT
