"""FP64 N-body oracle (Python side) — test infrastructure only (see ``oracle/__init__``).

Wraps the plain-C direct sum in ``nbody_ref.c`` (Section 4, N-Body on the Loop
skeleton). Conventions of the executor's N-body workload:

* state: x = float32 [N, 4] (position, mass), v and a = float32 [N, 4] with the
  4th slot unused; the oracle widens the float32 inputs to float64 and works
  in float64 throughout;
* G = 1 / N (the paper gives no constant; this keeps the mean field the same
  for every N), Plummer softening eps = 1e-3, dt = 1e-3;
* kick-drift-kick leapfrog; a Loop of k iterations is k such steps, and the
  acceleration is carried between steps, never recomputed at the start.

Pins: see ``nbody_ref.c``. Error metrics follow the workload's 1e-4 bound:
positions max_i |x_i - x^_i| / |x^_i|, velocities max_i |v_i - v^_i| / max_j |v^_j|.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

EPS = 1e-3
DT = 1e-3

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_nbody_accel.argtypes = [ctypes.c_int64, dp, ctypes.c_double, ctypes.c_double, dp, ctypes.c_int]
        lib.oracle_nbody_accel.restype = ctypes.c_int
        lib.oracle_nbody_kdk.argtypes = [ctypes.c_int64, dp, dp, dp, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int64, ctypes.c_int]
        lib.oracle_nbody_kdk.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def gravity(n: int) -> float:
    return 1.0 / n


def accel(x4: np.ndarray, g: float, eps: float = EPS, threads: int | None = None) -> np.ndarray:
    """[N, 3] float64 accelerations of the bodies in x4 ([N, 4]: position, mass)."""
    x = np.ascontiguousarray(x4, dtype=np.float64)
    n = x.shape[0]
    a = np.zeros((n, 3), dtype=np.float64)
    rc = _load().oracle_nbody_accel(n, _ptr(x), g, eps, _ptr(a), threads or default_threads())
    if rc:
        raise RuntimeError("oracle_nbody_accel failed")
    return a


def kdk(x4: np.ndarray, v: np.ndarray, a: np.ndarray, steps: int, g: float, eps: float = EPS, dt: float = DT,
        threads: int | None = None):
    """Return (x4, v, a) float64 after `steps` kick-drift-kick steps; `a` must be a(x) on entry."""
    x = np.array(x4, dtype=np.float64, order="C", copy=True)
    vv = np.array(np.asarray(v)[:, :3], dtype=np.float64, order="C", copy=True)
    aa = np.array(np.asarray(a)[:, :3], dtype=np.float64, order="C", copy=True)
    rc = _load().oracle_nbody_kdk(x.shape[0], _ptr(x), _ptr(vv), _ptr(aa), g, eps, dt, steps,
                                  threads or default_threads())
    if rc:
        raise RuntimeError("oracle_nbody_kdk failed")
    return x, vv, aa


def simulate(x4: np.ndarray, steps: int, g: float | None = None, eps: float = EPS, dt: float = DT,
             threads: int | None = None):
    """Pipeline(accel, Loop(kdk, steps)) from rest: returns (x4, v, a) in float64."""
    n = x4.shape[0]
    g = gravity(n) if g is None else g
    a0 = accel(x4, g, eps, threads)
    v0 = np.zeros((n, 3))
    return kdk(x4, v0, a0, steps, g, eps, dt, threads)


def accel_of(x4: np.ndarray, idx, g: float, eps: float = EPS) -> np.ndarray:
    """Accelerations of the bodies `idx` only (FP64, index-order sum), for sampled checks."""
    x = np.asarray(x4, dtype=np.float64)
    out = np.zeros((len(idx), 3))
    for k, i in enumerate(idx):
        d = x[:, :3] - x[i, :3]
        r2 = np.einsum("ij,ij->i", d, d) + eps * eps
        s = x[:, 3] / (r2 * np.sqrt(r2))
        out[k] = g * (s[:, None] * d).sum(axis=0)
    return out


def momentum(x4: np.ndarray, v: np.ndarray) -> np.ndarray:
    return (np.asarray(x4, dtype=np.float64)[:, 3:4] * np.asarray(v, dtype=np.float64)[:, :3]).sum(axis=0)


def pos_rel_error(x_test: np.ndarray, x_ref: np.ndarray) -> float:
    d = np.linalg.norm(np.asarray(x_test, np.float64)[:, :3] - np.asarray(x_ref, np.float64)[:, :3], axis=1)
    return float((d / np.linalg.norm(np.asarray(x_ref, np.float64)[:, :3], axis=1)).max())


def vel_rel_error(v_test: np.ndarray, v_ref: np.ndarray) -> float:
    vr = np.asarray(v_ref, np.float64)[:, :3]
    d = np.linalg.norm(np.asarray(v_test, np.float64)[:, :3] - vr, axis=1)
    return float(d.max() / max(np.linalg.norm(vr, axis=1).max(), 1e-300))
