"""Write the FP64 N-body reference trajectory end state used by the full-size GPU parity test.

Calls only the oracle (oracle.nbody) on the seeded input of paper_1510_06585_gb300.inputs:
N = 65536 bodies (seed 4), G = 1/N, eps = 1e-3, dt = 1e-3, 100 kick-drift-kick steps
(Section 4, N-Body on the Loop skeleton). The oracle is stepped one kick-drift-kick step per call
(the acceleration is carried between calls, so the result is bit-identical to one 100-step call),
and after every step the distance of each body to its nearest neighbour is taken
(scipy.spatial.cKDTree), so that the test can tell the bodies that passed inside a few softening
lengths of another body from the rest.

Stores, for every body, the final position and velocity (float64) and the smallest
nearest-neighbour distance over the 101 states (float64), plus the total momentum, in
nbody_65536_100steps.npz. Run: python tests/golden/make_nbody_golden.py
"""
import os
import sys

import numpy as np
from scipy.spatial import cKDTree

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import nbody  # noqa: E402
from paper_1510_06585_gb300 import inputs  # noqa: E402

N, STEPS = 65536, 100
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "nbody_65536_100steps.npz")


def nearest(x4):
    p = np.asarray(x4, np.float64)[:, :3]
    d, _ = cKDTree(p).query(p, k=2)
    return d[:, 1]


def main():
    x, _, _ = inputs.nbody(N, seed=inputs.SEED_NBODY)
    g = nbody.gravity(N)
    xs = np.asarray(x, np.float64)
    vs = np.zeros((N, 3))
    acc = nbody.accel(x, g)
    min_sep = nearest(xs)
    for s in range(STEPS):
        xs, vs, acc = nbody.kdk(xs, vs, acc, 1, g)
        min_sep = np.minimum(min_sep, nearest(xs))
        print(f"step {s + 1}/{STEPS}", flush=True)
    np.savez_compressed(OUT, x=xs[:, :3], v=vs, min_sep=min_sep, momentum=nbody.momentum(xs, vs),
                        meta=np.array([N, STEPS, inputs.SEED_NBODY, nbody.EPS, nbody.DT]))


if __name__ == "__main__":
    main()
