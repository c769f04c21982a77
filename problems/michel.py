"""Michel spherical accretion onto a Schwarzschild black hole (M = 1), as
initial data in Kerr-Schild coordinates with a = 0.

The steady, spherically symmetric, adiabatic inflow of a polytrope
p = K rho^Gamma is fixed by two constants of motion and one sonic point
(Michel 1972; e.g. Hawley, Smarr & Wilson 1984):
  mass flux   rho u^r r^2 = C1,
  Bernoulli   h^2 (1 - 2/r + (u^r)^2) = C2,          h = 1 + Gamma/(Gamma-1) p/rho,
and at the critical radius r_c the flow speed equals the sound speed:
  (u^r_c)^2 = 1 / (2 r_c),   c_s^2(r_c) = (u^r_c)^2 / (1 - 3 (u^r_c)^2),
with c_s^2 = Gamma p / (rho h).  The accretion branch is subsonic outside r_c
and supersonic inside; u^r is the same radial four-velocity component in
Schwarzschild and Kerr-Schild coordinates.
"""
from __future__ import annotations

import math

import numpy as np

from . import Grid, cell_centres, empty_prims

__all__ = ["michel_2d", "michel_constants", "michel_state", "michel_prims"]


def michel_2d(nblock=16, nroot=(4, 1), rmin=1.8, rmax=40.0, **kw) -> Grid:
    """Axisymmetric (r, theta) MKS grid, x1 = ln r from inside the horizon,
    theta in [pi/4, 3pi/4] (x2 in [0.25, 0.75]); outflow boundaries in both
    directions (the flow is spherically symmetric, so zero theta-gradient is
    exact), Gamma = 4/3, floors far below the flow."""
    g = Grid(ndim=2, nx=(nblock, nblock, 1), nroot=(nroot[0], nroot[1], 1),
             xmin=(math.log(rmin), 0.25, 0.0), xmax=(math.log(rmax), 0.75, 2.0 * math.pi),
             coords="mks", spin=0.0, mass=1.0,
             bc=(("outflow", "outflow"), ("outflow", "outflow"), ("periodic", "periodic")),
             recon="ppm", riemann="hll", gamma_ad=4.0 / 3.0, cfl=0.4, ch=1.0, kappa=0.1,
             rho_floor=1e-12, rho_floor_pow=0.0, p_floor=1e-14, p_floor_pow=0.0, w_max=50.0,
             name="michel_2d")
    return g.with_(**kw) if kw else g


def michel_constants(gam=4.0 / 3.0, r_c=8.0, rho_c=1e-2):
    """(K, C1, C2, n) of the flow through the sonic point r_c with density rho_c."""
    n = 1.0 / (gam - 1.0)
    uc2 = 1.0 / (2.0 * r_c)
    cs2 = uc2 / (1.0 - 3.0 * uc2)
    theta_c = cs2 / (gam - (n + 1.0) * cs2)     # p/rho at r_c, from c_s^2 = Gamma theta / (1 + (n+1) theta)
    K = theta_c / rho_c ** (gam - 1.0)
    C1 = rho_c * (-math.sqrt(uc2)) * r_c * r_c
    C2 = (1.0 + (n + 1.0) * theta_c) ** 2 * (1.0 - 2.0 / r_c + uc2)
    return K, C1, C2, n


def michel_state(r, gam=4.0 / 3.0, r_c=8.0, rho_c=1e-2):
    """rho, p and u^r (< 0) at radius r on the accretion branch."""
    from scipy.optimize import brentq
    K, C1, C2, n = michel_constants(gam, r_c, rho_c)

    def F(lth):  # Bernoulli residual in ln(theta), theta = p/rho
        th = math.exp(lth)
        rho = (th / K) ** n
        u = C1 / (rho * r * r)
        return (1.0 + (n + 1.0) * th) ** 2 * (1.0 - 2.0 / r + u * u) - C2

    # F has one minimum in ln(theta) (zero at r_c); the subsonic root lies
    # above it (outside r_c), the supersonic one below it (inside r_c)
    from scipy.optimize import minimize_scalar
    lo, hi = math.log(1e-12), math.log(10.0)
    lmin = minimize_scalar(F, bounds=(lo, hi), method="bounded", options={"xatol": 1e-13}).x
    if not F(lmin) < 0.0:
        lth = lmin  # at the sonic point the two roots meet
    elif r > r_c:
        lth = brentq(F, lmin, hi, xtol=1e-15, rtol=1e-15)
    else:
        lth = brentq(F, lo, lmin, xtol=1e-15, rtol=1e-15)
    th = math.exp(lth)
    rho = (th / K) ** n
    return rho, K * rho ** gam, C1 / (rho * r * r)


def michel_prims(grid: Grid, r_c=8.0, rho_c=1e-2) -> np.ndarray:
    """Code primitives of the Michel flow on a Kerr-Schild (a = 0) MKS grid:
    u^i(code) = u^i + u^t beta^i in (ln r, theta/pi, phi) components, with u^t
    the future-directed root of the Kerr-Schild normalisation
    -(1 - 2/r) (u^t)^2 + (4/r) u^t u^r + (1 + 2/r) (u^r)^2 = -1
    (written as 2C / (-B + sqrt(B^2 - 4AC)), regular across the horizon)."""
    assert grid.coords == "mks" and grid.spin == 0.0
    x1 = cell_centres(grid)[0]
    r = np.exp(x1)
    P = empty_prims(grid)
    radii = np.unique(r)
    table = {float(q): michel_state(float(q), grid.gamma_ad, r_c, rho_c) for q in radii}
    rho = np.vectorize(lambda q: table[float(q)][0])(r)
    p = np.vectorize(lambda q: table[float(q)][1])(r)
    ur = np.vectorize(lambda q: table[float(q)][2])(r)
    A = -(1.0 - 2.0 / r)
    B = 4.0 / r * ur
    C = (1.0 + 2.0 / r) * ur * ur + 1.0
    ut = 2.0 * C / (-B + np.sqrt(B * B - 4.0 * A * C))
    beta_r = (2.0 / r) / (1.0 + 2.0 / r)
    P[:, 0] = rho
    P[:, 1] = p
    P[:, 2] = (ur + ut * beta_r) / r   # d(ln r)/dr = 1/r
    return P
