"""Seeded synthetic inputs shared by the oracle's tests and the CUDA path.

This package holds problem set-ups only: grid records (sizes, boundary kinds,
scheme parameters) and initial primitive fields.  It contains none of the
finite-volume update's arithmetic, and neither the oracle nor the CUDA path
imports anything else from the other.

Primitive layout everywhere: ``prims[block, var, k, j, i]`` (interior cells,
``i`` fastest) with variables ``rho, p, u^1, u^2, u^3, B^1, B^2, B^3, psi`` and
``u^i = W v^i`` in code-coordinate components.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

NV = 9
SEED = 20210827


@dataclass
class Grid:
    ndim: int
    nx: tuple                 # interior cells per block (1 in inactive dimensions)
    nroot: tuple              # level-0 blocks per dimension
    xmin: tuple
    xmax: tuple
    coords: str = "cart"      # "cart", "ks" or "mks"
    spin: float = 0.0
    mass: float = 1.0
    bc: tuple = (("periodic", "periodic"),) * 3
    recon: str = "ppm"        # "ppm" or "minmod"
    riemann: str = "hll"      # "hll" or "tvdlf"
    gamma_ad: float = 4.0 / 3.0
    cfl: float = 0.4
    ch: float = 1.0
    kappa: float = 1.0
    c2p_tol: float = 1e-12
    c2p_maxit: int = 50
    rho_floor: float = 1e-12
    rho_floor_pow: float = 0.0
    p_floor: float = 1e-14
    p_floor_pow: float = 0.0
    w_max: float = 50.0
    divb: str = "glm"         # "glm" (cleaning) or "ct" (staggered-mesh constrained transport)
    imex: bool = False        # cleaning damping as the implicit part of IMEX-SSP2(2,2,2)
    c2p: str = "newton"       # primary inversion: "newton" (analytic Jacobian) or "nk" (Jacobian-free Newton-Krylov)
    ng: int = 3
    nlevels: int = 1
    blocks: np.ndarray = field(default=None, repr=False)  # (nb, 4) int32: level, ix, iy, iz
    name: str = ""

    def __post_init__(self):
        if self.blocks is None:
            self.blocks = uniform_blocks(self.nroot)

    @property
    def nb(self) -> int:
        return int(self.blocks.shape[0])

    @property
    def cells_per_block(self) -> int:
        return int(self.nx[0] * self.nx[1] * self.nx[2])

    @property
    def ncells(self) -> int:
        return self.nb * self.cells_per_block

    def with_(self, **kw) -> "Grid":
        return replace(self, **kw)


def uniform_blocks(nroot) -> np.ndarray:
    """All level-0 blocks, x fastest."""
    out = []
    for iz in range(nroot[2]):
        for iy in range(nroot[1]):
            for ix in range(nroot[0]):
                out.append((0, ix, iy, iz))
    return np.asarray(out, dtype=np.int32).reshape(-1, 4)


def cell_centres(grid: Grid):
    """Code coordinates of all interior cell centres, each (nb, nz, ny, nx)."""
    nb = grid.nb
    out = []
    for d in range(3):
        lev = grid.blocks[:, 0].astype(np.int64)
        scale = (2 ** lev) if d < grid.ndim else np.ones_like(lev)
        dx = (grid.xmax[d] - grid.xmin[d]) / (grid.nroot[d] * grid.nx[d] * scale)
        idx = np.arange(grid.nx[d])
        g = grid.blocks[:, 1 + d].astype(np.int64)[:, None] * grid.nx[d] + idx[None, :]
        x = grid.xmin[d] + (g + 0.5) * dx[:, None]
        shape = [nb, 1, 1, 1]
        shape[3 - d] = grid.nx[d]
        out.append(np.broadcast_to(x.reshape(shape), (nb, grid.nx[2], grid.nx[1], grid.nx[0])).copy())
    return out


def empty_prims(grid: Grid) -> np.ndarray:
    return np.zeros((grid.nb, NV, grid.nx[2], grid.nx[1], grid.nx[0]))


from .configs import *  # noqa: E402,F401,F403
from .flat import *  # noqa: E402,F401,F403
from .torus import *  # noqa: E402,F401,F403
from .michel import *  # noqa: E402,F401,F403
from .monopole import *  # noqa: E402,F401,F403
