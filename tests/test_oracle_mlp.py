"""Pins of the FP64 cost-model MLP oracle (no GPU)."""
import numpy as np
import pytest

from oracle import mlp as M


def _setup(k=5, n=7, seed=0):
    p = {kk: v.astype(np.float64) for kk, v in M.init_params(k, seed=seed).items()}
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    for kk in ("b1", "b2", "b3"):
        p[kk] = rng.normal(0, 0.1, size=p[kk].shape)
    x = rng.normal(size=(n, 16))
    t = rng.normal(size=(n, k))
    return p, x, t


def test_gradients_match_central_differences():
    p, x, t = _setup()
    g = M.backward(p, x, t)
    h = 1e-6
    rng = np.random.Generator(np.random.PCG64(3))
    for name in M.PARAM_NAMES:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = M.loss(p, x, t)
            flat[idx] = old - h
            lm = M.loss(p, x, t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, an)


def test_forward_matches_torch_linear_layers():
    torch = pytest.importorskip("torch")
    p, x, _ = _setup()
    y, _ = M.forward(p, x)
    tx = torch.tensor(x)
    h = torch.relu(torch.nn.functional.linear(tx, torch.tensor(p["w1"]), torch.tensor(p["b1"])))
    h = torch.relu(torch.nn.functional.linear(h, torch.tensor(p["w2"]), torch.tensor(p["b2"])))
    ty = torch.nn.functional.linear(h, torch.tensor(p["w3"]), torch.tensor(p["b3"]))
    assert np.allclose(y, ty.numpy(), rtol=1e-12, atol=1e-12)


def test_first_adam_step_closed_form():
    p, x, t = _setup()
    g = M.backward(p, x, t)
    zeros = {k: np.zeros_like(v) for k, v in p.items()}
    lr, eps = 1e-3, 1e-8
    w, m, v = M.adam_step(p, g, zeros, zeros, 1, lr, eps=eps)
    for k in M.PARAM_NAMES:
        # after one step m_hat = g and v_hat = g^2
        assert np.allclose(w[k], p[k] - lr * g[k] / (np.abs(g[k]) + eps), rtol=0, atol=1e-15)


def test_bf16_rounding_ties_to_even_like_torch():
    torch = pytest.importorskip("torch")
    vals = np.array([1.0, 0.5, -3.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, 65504.0, 1e-20, -7.3],
                    np.float32)
    r = M.bf16_round(vals)
    assert r[0] == 1.0 and r[3] == 1.0 and r[4] == np.float32(1 + 2 ** -6)
    want = torch.tensor(vals).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(r, want)
    rng = np.random.Generator(np.random.PCG64(0))
    many = rng.normal(size=10000).astype(np.float32) * 10.0 ** rng.integers(-8, 8, size=10000)
    assert np.array_equal(M.bf16_round(many), torch.tensor(many).to(torch.bfloat16).to(torch.float32).numpy())


def test_regret_definition():
    assert np.allclose(M.regret([1.1, 2.0], [1.0, 2.0]), [0.1, 0.0])
