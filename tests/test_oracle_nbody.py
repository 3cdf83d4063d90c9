"""Pins of the FP64 N-body oracle against closed forms and invariants (no GPU)."""
import math

import numpy as np

from oracle import nbody as O
from paper_1510_06585_gb300 import inputs


def test_two_body_closed_form():
    d, eps, g = 0.3, 0.05, 0.7
    x = np.array([[0.1, 0.2, 0.3, 1.0], [0.1 + d, 0.2, 0.3, 2.0]])
    a = O.accel(x, g, eps)
    mag = g / (d * d + eps * eps) ** 1.5 * d
    assert np.allclose(a[0], [2.0 * mag, 0, 0], rtol=1e-14, atol=0)
    assert np.allclose(a[1], [-1.0 * mag, 0, 0], rtol=1e-14, atol=0)


def test_single_body_feels_nothing():
    a = O.accel(np.array([[0.5, 0.5, 0.5, 3.0]]), 1.0, 1e-3)
    assert np.array_equal(a, np.zeros((1, 3)))


def test_cube_corners_point_to_centre_with_equal_magnitude():
    c = np.array([[i, j, k, 1.0] for i in (0, 1) for j in (0, 1) for k in (0, 1)], dtype=np.float64)
    a = O.accel(c, 1.0, 1e-3)
    mags = np.linalg.norm(a, axis=1)
    assert np.allclose(mags, mags[0], rtol=1e-13)
    to_centre = 0.5 - c[:, :3]
    cos = (a * to_centre).sum(axis=1) / (mags * np.linalg.norm(to_centre, axis=1))
    assert np.allclose(cos, 1.0, atol=1e-13)


def _accel_brute(x, g, eps):
    n = len(x)
    out = []
    for i in range(n):
        ax = ay = az = 0.0
        for j in range(n):
            dx, dy, dz = (x[j][k] - x[i][k] for k in range(3))
            r2 = dx * dx + dy * dy + dz * dz + eps * eps
            s = x[j][3] / r2 ** 1.5
            ax += s * dx
            ay += s * dy
            az += s * dz
        out.append([g * ax, g * ay, g * az])
    return np.array(out)


def test_brute_force_small_n():
    for n in (2, 3, 8, 16):
        x, _, _ = inputs.nbody(n, seed=n)
        xx = x.astype(np.float64).tolist()
        assert np.allclose(O.accel(x, 1.0 / n, 1e-3), _accel_brute(xx, 1.0 / n, 1e-3), rtol=1e-12, atol=1e-14)


def test_sampled_accel_helper_matches_full_sum():
    x, _, _ = inputs.nbody(300, seed=1)
    idx = [0, 17, 299]
    assert np.allclose(O.accel_of(x, idx, 1 / 300), O.accel(x, 1 / 300)[idx], rtol=1e-12)


def test_momentum_conserved_by_forces_and_integrator():
    x, _, _ = inputs.nbody(257, seed=3)
    g = 1.0 / 257
    a = O.accel(x, g)
    f = (x[:, 3:4].astype(np.float64) * a).sum(axis=0)
    assert np.linalg.norm(f) <= 1e-12 * (x[:, 3:4] * np.abs(a)).sum()
    xs, vs, _ = O.simulate(x, 20)
    p = O.momentum(xs, vs)
    assert np.linalg.norm(p) <= 1e-12 * (xs[:, 3:4] * np.abs(vs)).sum()


def test_loop_k_equals_k_single_steps():
    x, _, _ = inputs.nbody(64, seed=5)
    g = 1 / 64
    a0 = O.accel(x, g)
    v0 = np.zeros((64, 3))
    x7, v7, a7 = O.kdk(x, v0, a0, 7, g)
    xa, va, aa = O.kdk(x, v0, a0, 3, g)
    xb, vb, ab = O.kdk(xa, va, aa, 4, g)
    assert np.array_equal(x7, xb) and np.array_equal(v7, vb) and np.array_equal(a7, ab)


def _circular_orbit_error(steps_per_period):
    # two unit masses a distance 1 apart, G = 1, negligible softening (the j = i term needs eps > 0):
    # each moves on a circle of radius r = 1/2; m v^2 / r = G m m / d^2 with d = 1 gives v = sqrt(0.5)
    v0 = math.sqrt(0.5)
    period = 2 * math.pi * 0.5 / v0
    x = np.array([[-0.5, 0, 0, 1.0], [0.5, 0, 0, 1.0]])
    v = np.array([[0, -v0, 0], [0, v0, 0]], dtype=np.float64)
    dt = period / steps_per_period
    a = O.accel(x, 1.0, 1e-9)
    xe, _, _ = O.kdk(x, v, a, steps_per_period, 1.0, 1e-9, dt)
    return np.linalg.norm(xe[:, :3] - x[:, :3], axis=1).max()


def test_kick_drift_kick_is_second_order():
    e1 = _circular_orbit_error(200)
    e2 = _circular_orbit_error(400)
    assert e1 < 1e-2
    assert 3.0 < e1 / e2 < 5.0


def test_error_metrics():
    x = np.array([[1.0, 0, 0, 1], [0, 2.0, 0, 1]])
    y = x.copy()
    y[1, 1] += 2e-4
    assert abs(O.pos_rel_error(y, x) - 1e-4) < 1e-12
