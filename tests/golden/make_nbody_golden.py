"""Write the FP64 N-body reference trajectory sample used by the full-size GPU parity test.

Calls only the oracle (oracle.nbody) on the seeded input of paper_1510_06585_gb300.inputs:
N = 65536 bodies (seed 4), G = 1/N, eps = 1e-3, dt = 1e-3, 100 kick-drift-kick steps
(Section 4, N-Body on the Loop skeleton). Stores every 64th body's final position and velocity
and the total momentum. Run: python tests/golden/make_nbody_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import nbody  # noqa: E402
from paper_1510_06585_gb300 import inputs  # noqa: E402

N, STEPS, STRIDE = 65536, 100, 64
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "nbody_65536_100steps.txt")


def main():
    x, _, _ = inputs.nbody(N, seed=inputs.SEED_NBODY)
    xs, vs, _ = nbody.simulate(x, STEPS)
    p = nbody.momentum(xs, vs)
    with open(OUT, "w") as f:
        f.write("# FP64 oracle (oracle/nbody_ref.c), N=65536 seed=4, G=1/N, eps=1e-3, dt=1e-3, 100 KDK steps\n")
        f.write("# written by tests/golden/make_nbody_golden.py; every 64th body: i x y z vx vy vz\n")
        f.write("# momentum %.17g %.17g %.17g\n" % tuple(p))
        for i in range(0, N, STRIDE):
            f.write("%d %.17g %.17g %.17g %.17g %.17g %.17g\n" % (i, *xs[i, :3], *vs[i, :3]))


if __name__ == "__main__":
    main()
