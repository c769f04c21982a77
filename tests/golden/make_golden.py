"""Writes the stored oracle fixtures of tests/golden/ (calls only oracle/ and
the seeded inputs; run from the repository root: python -m tests.golden.make_golden).

shock_tube_profile.txt: the 2-D shock tube (128x128 cells as 16 blocks of 32x32,
Gamma = 2, PPM + HLL, CFL 0.4, GLM) after 100 steps; row j = 0 of the
primitives along x, one line per cell: rho p u1 u2 u3 B1 B2 B3 psi.
The paper prints no reference solution for this problem; the file only
guards the oracle against unintended changes."""
import os

import numpy as np

import oracle
import problems as pb

HERE = os.path.dirname(os.path.abspath(__file__))


def shock_tube_profile(steps=100):
    g = pb.shock_tube_2d()
    o = oracle.Oracle(g)
    o.set_prims(pb.shock_tube_prims(g))
    for _ in range(steps):
        o.step(o.cfl_dt())
    Q = o.prims()
    return np.concatenate([Q[b, :, 0, 0, :] for b in range(4)], axis=1).T


if __name__ == "__main__":
    np.savetxt(os.path.join(HERE, "shock_tube_profile.txt"), shock_tube_profile(), fmt="%.17e")
