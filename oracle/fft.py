"""Oracle for the FFT pipeline stages — test infrastructure only (see ``oracle/__init__``).

Section 4 of the paper (FFT benchmark): SHOC-derived fast Fourier transforms, each followed in a
Pipeline by the inverse transform; one transform of 512 KB (65,536 single-precision complex values)
is the unit the data is partitioned by. The transforms are the discrete Fourier transform and
its inverse, applied to every row of an (nfft, N) complex array:

* fft  : X[k] = sum_n x[n] exp(-2 pi i n k / N)            (forward, not normalised)
* ifft : x[n] = (1 / N) sum_k X[k] exp(+2 pi i n k / N)    (inverse, normalised by 1 / N)

The paper does not state the normalisation; the inverse carries the 1 / N so that the pipelined
pair returns its input. Each stage is a library FFT (numpy.fft, complex128) on the float32 inputs
widened to float64, stages applied one after another with every intermediate materialised.

Pins (tests/test_oracle_fft.py): an explicit O(N^2) sum on small N; the transform of a unit impulse
(all ones), of a constant (N at index 0) and of a complex exponential exp(2 pi i k0 n / N) (N at
index k0, which fixes the sign convention); the shift theorem; Parseval's identity (which fixes the
forward transform's lack of normalisation); the inverse of the transform; fft(fft(x))[n] =
N x[-n mod N].
"""
from __future__ import annotations

import numpy as np


def fft_rows(x: np.ndarray) -> np.ndarray:
    """Forward DFT of every row (last axis), complex128."""
    return np.fft.fft(np.asarray(x, dtype=np.complex128), axis=-1)


def ifft_rows(x: np.ndarray) -> np.ndarray:
    """Inverse DFT (normalised by 1 / N) of every row (last axis), complex128."""
    return np.fft.ifft(np.asarray(x, dtype=np.complex128), axis=-1)


def pipeline(x: np.ndarray, stages) -> np.ndarray:
    """Apply the stages ("fft" / "ifft") in order, each on the previous stage's whole output."""
    y = np.asarray(x, dtype=np.complex128)
    for s in stages:
        if s == "fft":
            y = fft_rows(y)
        elif s == "ifft":
            y = ifft_rows(y)
        else:
            raise ValueError(f"unknown FFT stage {s!r}")
    return y


def rel_error(got: np.ndarray, want: np.ndarray) -> float:
    """Largest per-row normwise relative error ||got - want|| / ||want|| over the rows."""
    got = np.asarray(got, dtype=np.complex128).reshape(-1, np.shape(want)[-1])
    want = np.asarray(want, dtype=np.complex128).reshape(got.shape)
    num = np.linalg.norm(got - want, axis=-1)
    den = np.linalg.norm(want, axis=-1)
    return float((num / np.maximum(den, 1e-300)).max())
