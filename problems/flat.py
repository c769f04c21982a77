"""Flat-space (Minkowski, Cartesian) initial data."""
from __future__ import annotations

import math

import numpy as np

from . import NV, SEED, Grid, cell_centres, empty_prims

__all__ = ["shock_tube_prims", "contact_wave_prims", "alfven_wave_prims", "alfven_speed",
           "random_periodic_prims"]


def shock_tube_prims(grid: Grid) -> np.ndarray:
    """Two states separated at x = 0.5: (rho, p, Bx, By) = (1, 1, 0.5, 1) on the
    left and (0.125, 0.1, 0.5, -1) on the right, at rest, psi = 0."""
    x, _, _ = cell_centres(grid)
    P = empty_prims(grid)
    left = x < 0.5
    P[:, 0] = np.where(left, 1.0, 0.125)
    P[:, 1] = np.where(left, 1.0, 0.1)
    P[:, 5] = 0.5
    P[:, 6] = np.where(left, 1.0, -1.0)
    return P


def contact_wave_prims(grid: Grid, t: float = 0.0, v: float = 0.5, amp: float = 0.5, p: float = 1.0,
                       bx: float = 0.5) -> np.ndarray:
    """Density wave rho = 1 + amp sin(2 pi (x - v t)) in uniform velocity v,
    pressure p and field B = (bx, 0, 0) parallel to v: an exact contact wave."""
    x, _, _ = cell_centres(grid)
    P = empty_prims(grid)
    W = 1.0 / math.sqrt(1.0 - v * v)
    P[:, 0] = 1.0 + amp * np.sin(2.0 * np.pi * (x - v * t))
    P[:, 1] = p
    P[:, 2] = W * v
    P[:, 5] = bx
    return P


def alfven_speed(rho: float, p: float, gamma_ad: float, b0: float, eta: float) -> float:
    """Propagation speed of the large-amplitude circularly polarised Alfven
    wave of relativistic MHD (Del Zanna, Zanotti, Landi & Bucciantini 2007):
      v_A^2 = 2 B0^2 / ((rho h + B0^2 (1 + eta^2)) (1 + sqrt(1 - (2 eta B0^2 / (rho h + B0^2 (1 + eta^2)))^2)))."""
    rhoh = rho + gamma_ad / (gamma_ad - 1.0) * p
    e = rhoh + b0 * b0 * (1.0 + eta * eta)
    return math.sqrt(2.0 * b0 * b0 / (e * (1.0 + math.sqrt(1.0 - (2.0 * eta * b0 * b0 / e) ** 2))))


def alfven_wave_prims(grid: Grid, t: float = 0.0, rho: float = 1.0, p: float = 1.0, b0: float = 1.0,
                      eta: float = 1.0) -> np.ndarray:
    """Circularly polarised Alfven wave along x with wavelength 1:
    B = (B0, eta B0 cos(k(x - vA t)), eta B0 sin(k(x - vA t))), v = -vA B_t / B0."""
    x, _, _ = cell_centres(grid)
    vA = alfven_speed(rho, p, grid.gamma_ad, b0, eta)
    ph = 2.0 * np.pi * (x - vA * t)
    by, bz = eta * b0 * np.cos(ph), eta * b0 * np.sin(ph)
    vy, vz = -vA * by / b0, -vA * bz / b0
    W = 1.0 / np.sqrt(1.0 - vy * vy - vz * vz)
    P = empty_prims(grid)
    P[:, 0] = rho
    P[:, 1] = p
    P[:, 3] = W * vy
    P[:, 4] = W * vz
    P[:, 5] = b0
    P[:, 6] = by
    P[:, 7] = bz
    return P


def random_periodic_prims(grid: Grid, seed: int = SEED, jump: bool = True) -> np.ndarray:
    """Smooth periodic modes with random phases and amplitudes (plus, with
    ``jump``, a density and pressure step) for conservation checks."""
    rng = np.random.default_rng(seed)
    xs = cell_centres(grid)
    P = empty_prims(grid)

    def mode(scale):
        out = np.zeros_like(xs[0])
        for d in range(grid.ndim):
            k = rng.integers(1, 3)
            out += scale * rng.uniform(0.2, 1.0) * np.sin(2 * np.pi * k * xs[d] + rng.uniform(0, 2 * np.pi))
        return out

    P[:, 0] = 1.0 + 0.5 * np.tanh(mode(1.0))
    P[:, 1] = 1.0 + 0.5 * np.tanh(mode(1.0))
    for i in range(3):
        P[:, 2 + i] = mode(0.4)
    for i in range(3):
        P[:, 5 + i] = mode(0.5)
    P[:, 8] = mode(0.05)
    if jump:
        inside = (xs[0] - 0.5) ** 2 + ((xs[1] - 0.5) ** 2 if grid.ndim > 1 else 0.0) < 0.04
        P[:, 0] = np.where(inside, 3.0 * P[:, 0], P[:, 0])
        P[:, 1] = np.where(inside, 2.0 * P[:, 1], P[:, 1])
    return P
