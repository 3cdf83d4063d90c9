"""Pins of the Saxpy oracle (Section 4, Saxpy) against exact arithmetic."""
import numpy as np

from oracle import saxpy as S


def _ints(n, lo, hi, seed):
    return np.random.Generator(np.random.PCG64(seed)).integers(lo, hi, size=n).astype(np.float32)


def test_integer_inputs_give_the_closed_form():
    # every value below 2^53: float64 is exact, so k stages equal y0 + (sum of alphas) x
    x, y = _ints(1000, -1000, 1000, 1), _ints(1000, -1000, 1000, 2)
    alphas = [3.0, -2.0, 7.0, 0.5]
    got = S.saxpy_stages(x, y, alphas)
    want = y.astype(np.int64) * 2 + (3 * 2 - 2 * 2 + 7 * 2 + 1) * x.astype(np.int64)
    assert np.array_equal(got * 2, want.astype(np.float64))


def test_hand_worked_single_stage():
    got = S.saxpy_stages(np.array([1, 2, -3, 0.5], np.float32), np.array([10, 0, 1, -1], np.float32), [2.0])
    assert got.tolist() == [12.0, 4.0, -5.0, 0.0]


def test_identity_and_cancellation():
    rng = np.random.Generator(np.random.PCG64(3))
    x = rng.normal(size=257).astype(np.float32)
    y = rng.normal(size=257).astype(np.float32)
    assert np.array_equal(S.saxpy_stages(x, y, [0.0]), y.astype(np.float64))
    # integer-valued x: a x and -a x are exact, so a stage and its negation cancel exactly
    xi = _ints(257, -50, 50, 4)
    assert np.array_equal(S.saxpy_stages(xi, y, [1.25, -1.25]), y.astype(np.float64))


def test_stage_order_does_not_change_an_exact_result():
    x, y = _ints(300, -100, 100, 5), _ints(300, -100, 100, 6)
    assert np.array_equal(S.saxpy_stages(x, y, [1, 2, 3]), S.saxpy_stages(x, y, [3, 1, 2]))
    # and x, y are not interchangeable: a dropped or swapped operand shows
    assert not np.array_equal(S.saxpy_stages(x, y, [2.0]), S.saxpy_stages(y, x, [2.0]))


def test_alpha_is_rounded_to_float32_like_the_stage_parameter():
    x = np.ones(1, np.float32)
    assert S.saxpy_stages(x, np.zeros(1, np.float32), [0.1])[0] == float(np.float32(0.1))


def test_error_bound_covers_float32_rounding():
    rng = np.random.Generator(np.random.PCG64(7))
    x = rng.normal(size=4096).astype(np.float32)
    y = rng.normal(size=4096).astype(np.float32)
    alphas = [2.5, -1.5, 0.75]
    # float32 evaluation with one rounding per stage (float64 product and sum are exact here for
    # the sum, then rounded once to float32)
    yf = y.copy()
    for a in alphas:
        yf = (np.float64(np.float32(a)) * x.astype(np.float64) + yf.astype(np.float64)).astype(np.float32)
    err = np.abs(yf.astype(np.float64) - S.saxpy_stages(x, y, alphas))
    assert (err <= S.error_bound(x, y, alphas)).all()
    assert err.max() > 0  # the bound is exercised by real rounding
