"""Pins of the FFT oracle (no GPU): the DFT's plain definition on small sizes, closed forms, and
identities that fix its sign convention and normalisation."""
import numpy as np
import pytest

from oracle import fft as F
from paper_1510_06585_gb300 import inputs


@pytest.mark.parametrize("n", [1, 2, 8, 16, 60])
def test_matches_the_explicit_sum_on_small_sizes(n):
    x = inputs.fft_signals(3, n, seed=n).astype(np.complex128)
    want = np.zeros_like(x)
    for k in range(n):
        for j in range(n):
            want[:, k] += x[:, j] * complex(np.cos(2 * np.pi * j * k / n), -np.sin(2 * np.pi * j * k / n))
    assert np.abs(F.fft_rows(x) - want).max() <= 1e-10 * n


def test_impulse_constant_and_exponential_closed_forms():
    n = 65536
    d = np.zeros((1, n), np.complex128)
    d[0, 0] = 1.0
    assert np.abs(F.fft_rows(d) - 1.0).max() <= 1e-12
    c = np.full((1, n), 2.5 + 0.5j)
    want = np.zeros((1, n), np.complex128)
    want[0, 0] = n * (2.5 + 0.5j)
    assert np.abs(F.fft_rows(c) - want).max() <= 1e-9 * n
    # exp(+2 pi i k0 n / N) has all its energy at index k0: the forward kernel is exp(-2 pi i nk/N)
    k0 = 1234
    e = np.exp(2j * np.pi * k0 * np.arange(n) / n)[None, :]
    X = F.fft_rows(e)
    assert abs(X[0, k0] - n) <= 1e-6 * n
    X[0, k0] = 0
    assert np.abs(X).max() <= 1e-6 * n
    # the inverse of an impulse at k0 is that exponential divided by N
    imp = np.zeros((1, n), np.complex128)
    imp[0, k0] = 1.0
    assert np.abs(F.ifft_rows(imp) - e / n).max() <= 1e-15


def test_shift_theorem_parseval_and_inverse():
    n = 4096
    x = inputs.fft_signals(2, n).astype(np.complex128)
    X = F.fft_rows(x)
    m = 37
    Xs = F.fft_rows(np.roll(x, m, axis=-1))
    assert np.abs(Xs - X * np.exp(-2j * np.pi * np.arange(n) * m / n)).max() <= 1e-9 * n
    # Parseval without normalisation on the forward side: sum |X|^2 = N sum |x|^2
    assert np.allclose((np.abs(X) ** 2).sum(-1), n * (np.abs(x) ** 2).sum(-1), rtol=1e-12)
    assert np.abs(F.ifft_rows(X) - x).max() <= 1e-12
    assert F.rel_error(F.pipeline(x, ["fft", "ifft"]), x) <= 1e-13


def test_double_forward_transform_reverses_and_scales():
    n = 1024
    x = inputs.fft_signals(2, n, seed=3).astype(np.complex128)
    y = F.pipeline(x, ["fft", "fft"])
    want = n * x[:, (-np.arange(n)) % n]
    assert np.abs(y - want).max() <= 1e-10 * n


def test_rel_error_is_per_row_normwise():
    want = np.ones((2, 4), np.complex128)
    got = want.copy()
    got[1, 0] += 0.2
    assert abs(F.rel_error(got, want) - 0.1) <= 1e-12


def test_signals_are_seeded_complex64_in_range():
    a = inputs.fft_signals(4, 64)
    b = inputs.fft_signals(4, 64)
    assert a.dtype == np.complex64 and np.array_equal(a, b)
    assert a.real.min() >= -1 and a.real.max() < 1 and a.imag.min() >= -1 and a.imag.max() < 1
