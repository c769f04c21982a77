"""Named grids of the benchmark workloads and of the tests.

Workloads (sizes as stated for the method's benchmark):
  shock_tube_2d    2-D special-relativistic MHD shock tube, 128x128 cells as
                   16 blocks of 32x32, Gamma = 2, PPM + HLL, CFL 0.4, GLM.
  torus_2d         2-D axisymmetric Fishbone-Moncrief torus, Kerr a = 0.9375,
                   modified Kerr-Schild, 256x256 as 256 blocks of 16x16,
                   r in [1.2, 2500] log-spaced, theta in (0, pi), Gamma = 4/3.
  torus_3d         the same torus in 3-D, 192x96x96 cells as 432 blocks of 16^3.
  torus_3d_large   512x256x256 cells as 2048 blocks of 32x32x16 (and the same
                   grid in other block shapes for the block-size sweep).
"""
from __future__ import annotations

import math

from . import Grid

__all__ = ["shock_tube_2d", "torus_2d", "torus_3d", "torus_3d_large", "periodic_box", "amr_torus", "TORUS_SPIN"]

TORUS_SPIN = 0.9375
R_IN, R_OUT = 1.2, 2500.0


def shock_tube_2d(nblock=32, nroot=4, **kw) -> Grid:
    g = Grid(ndim=2, nx=(nblock, nblock, 1), nroot=(nroot, nroot, 1), xmin=(0.0, 0.0, 0.0),
             xmax=(1.0, 1.0, 1.0), coords="cart",
             bc=(("outflow", "outflow"), ("periodic", "periodic"), ("periodic", "periodic")),
             recon="ppm", riemann="hll", gamma_ad=2.0, cfl=0.4, ch=1.0, kappa=1.0,
             rho_floor=1e-12, p_floor=1e-14, name="shock_tube_2d")
    return g.with_(**kw) if kw else g


def _torus_common(ndim, nx, nroot, name, **kw) -> Grid:
    g = Grid(ndim=ndim, nx=nx, nroot=nroot,
             xmin=(math.log(R_IN), 0.0, 0.0), xmax=(math.log(R_OUT), 1.0, 2.0 * math.pi),
             coords="mks", spin=TORUS_SPIN, mass=1.0,
             bc=(("noinflow", "noinflow"), ("axis", "axis"), ("periodic", "periodic")),
             recon="ppm", riemann="hll", gamma_ad=4.0 / 3.0, cfl=0.4, ch=1.0, kappa=0.1,
             rho_floor=1e-5, rho_floor_pow=-1.5, p_floor=1e-7 / 3.0, p_floor_pow=-2.5,
             w_max=50.0, name=name)
    return g.with_(**kw) if kw else g


def torus_2d(nblock=16, nroot=(16, 16), **kw) -> Grid:
    return _torus_common(2, (nblock, nblock, 1), (nroot[0], nroot[1], 1), "torus_2d", **kw)


def torus_3d(nblock=(16, 16, 16), nroot=(12, 6, 6), **kw) -> Grid:
    return _torus_common(3, tuple(nblock), tuple(nroot), "torus_3d", **kw)


def torus_3d_large(nblock=(32, 32, 16), cells=(512, 256, 256), **kw) -> Grid:
    nroot = tuple(c // b for c, b in zip(cells, nblock))
    assert all(r * b == c for r, b, c in zip(nroot, nblock, cells))
    return _torus_common(3, tuple(nblock), nroot, "torus_3d_large", **kw)


def periodic_box(ndim=2, nblock=8, nroot=2, **kw) -> Grid:
    nx = tuple(nblock if d < ndim else 1 for d in range(3))
    nr = tuple(nroot if d < ndim else 1 for d in range(3))
    g = Grid(ndim=ndim, nx=nx, nroot=nr, xmin=(0.0, 0.0, 0.0), xmax=(1.0, 1.0, 1.0),
             coords="cart", bc=(("periodic", "periodic"),) * 3, gamma_ad=5.0 / 3.0, name="periodic_box")
    return g.with_(**kw) if kw else g


def amr_torus(root=(8, 4, 5), nblock=16, r_refine=(60.0, 20.0), **kw) -> Grid:
    """Three-level torus: root blocks of nblock^3 in MKS; a block is refined to
    level 1 where its inner radius is below r_refine[0] and, at level 1, to
    level 2 where its inner radius is below r_refine[1] (finest level inside
    r < 20 M).  Refinement depends on r only, so neighbouring blocks differ by
    at most one level across faces, edges and corners (and through the axis).
    Leaf blocks only, ordered by level then z, y, x."""
    x1min, x1max = math.log(R_IN), math.log(R_OUT)
    leaves = []

    def inner_r(level, ix):
        w = (x1max - x1min) / (root[0] * 2 ** level)
        return math.exp(x1min + ix * w)

    def visit(level, ix, iy, iz):
        if level < len(r_refine) and inner_r(level, ix) < r_refine[level]:
            for dz in (0, 1):
                for dy in (0, 1):
                    for dx in (0, 1):
                        visit(level + 1, 2 * ix + dx, 2 * iy + dy, 2 * iz + dz)
        else:
            leaves.append((level, ix, iy, iz))

    for iz in range(root[2]):
        for iy in range(root[1]):
            for ix in range(root[0]):
                visit(0, ix, iy, iz)
    import numpy as np
    blocks = np.asarray(sorted(leaves, key=lambda b: (b[0], b[3], b[2], b[1])), dtype=np.int32)
    g = _torus_common(3, (nblock, nblock, nblock), tuple(root), "amr_torus", **kw)
    return g.with_(nlevels=len(r_refine) + 1, blocks=blocks)
