"""GPU cost-model kernels against the FP64 oracle: forward, gradients, Adam, and training."""
import numpy as np
import pytest
import torch

from oracle import mlp as O
from paper_1510_06585_gb300 import mrw as M

pytestmark = pytest.mark.gpu

K, H = 16, 64


def _params(seed=0):
    p = O.init_params(K, hidden=H, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed + 10))
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(0, 0.1, size=p[k].shape).astype(np.float32)
    return p


def _data(n, seed=1):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.normal(size=(n, 16)).astype(np.float32), rng.normal(size=(n, K)).astype(np.float32)


def _rounded(p):
    return {k: O.bf16_round(v) for k, v in p.items()}


def test_forward_matches_oracle_on_bf16_weights():
    m = M.Model(K, H)
    p = _params()
    m.set_params(M.pack_params(p))
    x, _ = _data(300)
    y = torch.zeros(300, K, device="cuda")
    m.forward(torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    want, _ = O.forward(_rounded(p), x)
    assert np.abs(y.cpu().numpy() - want).max() <= 1e-4 * np.abs(want).max()


def test_gradients_match_oracle():
    m = M.Model(K, H)
    p = _params(3)
    m.set_params(M.pack_params(p))
    x, t = _data(257, seed=4)
    g = torch.zeros(m.num_params(), device="cuda")
    loss = m.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), g)
    pr = _rounded(p)
    want = O.backward(pr, x, t)
    got = M.unpack_params(g.cpu().numpy(), K, H)
    for k in O.PARAM_NAMES:
        err = np.linalg.norm(got[k] - want[k]) / max(np.linalg.norm(want[k]), 1e-30)
        assert err <= 1e-4, (k, err)
    assert abs(loss - O.loss(pr, x, t)) <= 1e-5 * O.loss(pr, x, t)


def test_adam_step_matches_oracle_and_refreshes_bf16():
    m = M.Model(K, H)
    p = _params(5)
    m.set_params(M.pack_params(p))
    rng = np.random.Generator(np.random.PCG64(6))
    grads = rng.normal(size=m.num_params()).astype(np.float32)
    gd = torch.from_numpy(grads).cuda()
    m.adam_step(gd, 1e-2)
    m.adam_step(gd, 1e-2)
    torch.cuda.synchronize()
    gp = M.unpack_params(grads, K, H)
    zeros = {k: np.zeros_like(v, dtype=np.float64) for k, v in p.items()}
    w, mm, vv = O.adam_step(p, gp, zeros, zeros, 1, 1e-2)
    w, mm, vv = O.adam_step(w, gp, mm, vv, 2, 1e-2)
    got = M.unpack_params(m.get_params(), K, H)
    for k in O.PARAM_NAMES:
        assert np.abs(got[k] - w[k]).max() <= 1e-6 + 1e-5 * np.abs(w[k]).max(), k
    # the forward pass now uses the bf16 rounding of the updated master weights
    x, _ = _data(64, seed=7)
    y = torch.zeros(64, K, device="cuda")
    m.forward(torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    want, _ = O.forward(_rounded({k: got[k].astype(np.float32) for k in got}), x)
    assert np.abs(y.cpu().numpy() - want).max() <= 1e-4 * np.abs(want).max()


def test_training_fits_a_smooth_target():
    rng = np.random.Generator(np.random.PCG64(8))
    x = rng.normal(size=(4096, 16)).astype(np.float32)
    wt = rng.normal(size=(16, K)).astype(np.float32) / 4
    t = np.tanh(x @ wt).astype(np.float32)
    m = M.Model(K, H, seed=1)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    first = m.train(xd, td, epochs=1, batch=128, lr=3e-3, seed=0)
    last = m.train(xd, td, epochs=60, batch=128, lr=3e-3, seed=1)
    assert last < 0.1 * first, (first, last)
