"""A static, force-free magnetic monopole in flat space in spherical
coordinates (Kerr-Schild coordinates with M = 0, a = 0): uniform density and
pressure, no flow, radial field B^r = B0/r^2 (curl-free, so the Lorentz force
vanishes), psi = 0.  It is an exact equilibrium of the continuum equations:
the magnetic pressure gradient is balanced by the hoop terms of the
curvilinear geometry."""
from __future__ import annotations

import math

from . import Grid, cell_centres, empty_prims

__all__ = ["monopole_flat_spherical", "monopole_prims"]


def monopole_flat_spherical(nr_blocks=2, nblock=16) -> Grid:
    """r in [2, 6], theta in [pi/4, 3pi/4] as nr_blocks x nr_blocks/2 blocks
    of nblock^2; zero-gradient (outflow) boundaries."""
    return Grid(ndim=2, nx=(nblock, nblock, 1), nroot=(nr_blocks, max(1, nr_blocks // 2), 1),
                xmin=(2.0, math.pi / 4, 0.0), xmax=(6.0, 3 * math.pi / 4, 2 * math.pi), coords="ks",
                spin=0.0, mass=0.0, bc=(("outflow", "outflow"), ("outflow", "outflow"), ("periodic", "periodic")),
                recon="ppm", riemann="hll", gamma_ad=4.0 / 3.0, ch=1.0, kappa=0.1, name="monopole_flat_spherical")


def monopole_prims(grid: Grid, rho=1.0, p=0.1, B0=4.0 * math.sqrt(0.1)):
    """Code primitives (B0 = 4 sqrt(0.1): B^2 = p at r = 2)."""
    r = cell_centres(grid)[0]
    P = empty_prims(grid)
    P[:, 0] = rho
    P[:, 1] = p
    P[:, 5] = B0 / r ** 2
    return P
