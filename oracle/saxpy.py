"""Saxpy Map oracle — test infrastructure only (see ``oracle/__init__``).

Section 4 of the paper, Saxpy: the single-precision a·x + y over two vectors, a plain Map with
no data dependences. A Map (or Pipeline, or Loop) of k saxpy stages applies them in order to the
same x: y_k = alpha_k · x + y_{k-1}. The oracle computes that definition in float64 from the
float32 inputs and the float32 alphas the stages hold (a stage's alpha is a float32 parameter),
one stage after another, every intermediate a full vector.

Pins (tests/test_oracle_saxpy.py): integer-valued inputs, where float64 is exact and the result
has the closed form y0 + (sum of alphas) · x; alpha = 0 is the identity; a stage and its negation
cancel exactly; the order of stages does not change an exact result; one stage against a
hand-worked vector.
"""
from __future__ import annotations

import numpy as np


def saxpy_stages(x: np.ndarray, y: np.ndarray, alphas) -> np.ndarray:
    """float64 y after applying y := alpha · x + y for each alpha in order (alpha rounded to
    float32, as the stage stores it)."""
    xd = np.asarray(x, dtype=np.float64)
    yd = np.array(y, dtype=np.float64, copy=True)
    for a in alphas:
        yd = float(np.float32(a)) * xd + yd
    return yd


def error_bound(x: np.ndarray, y: np.ndarray, alphas) -> np.ndarray:
    """Elementwise bound on |float32 result - saxpy_stages| for k stages each rounded once
    (a fused multiply-add per stage): every stage adds at most one rounding of its result, whose
    magnitude is at most |y0| + sum_k |alpha_k x|, so k · 2^-23 times that bounds the total
    (twice the unit roundoff per stage, which also covers the growth of earlier errors)."""
    xd = np.abs(np.asarray(x, dtype=np.float64))
    m = np.abs(np.asarray(y, dtype=np.float64)) + sum(abs(float(np.float32(a))) for a in alphas) * xd
    return len(list(alphas)) * 2.0 ** -23 * m
