"""Fishbone-Moncrief torus around a Kerr black hole (M = 1), in modified
Kerr-Schild code coordinates (x1 = ln r, x2 = theta / pi, x3 = phi).

Equilibrium (Fishbone & Moncrief 1976): a barotropic torus whose fluid has
u^t u_phi = l constant.  With the Boyer-Lindquist functions
  e^{2 nu} = Sigma Delta / A, e^{2 psi} = A sin^2 th / Sigma, omega = 2 a r / A,
the Euler equation integrates to
  ln h = 1/2 ln((1 + s) / e^{2 nu}) - s/2 - l omega + const,
  s = sqrt(1 + 4 l^2 e^{2 nu} / e^{2 psi}),
with the constant fixed by h = 1 at the inner edge (r_in, pi/2) and l fixed by
putting the pressure maximum at r_pmax in the equatorial plane.
"""
from __future__ import annotations

import math

import numpy as np

from . import NV, SEED, Grid, cell_centres, empty_prims

__all__ = ["fm_constants", "fm_lnh", "fm_torus_prims", "ks_code_metric"]


def _bl(r, th, a):
    s2 = np.sin(th) ** 2
    Sigma = r * r + a * a * np.cos(th) ** 2
    Delta = r * r - 2.0 * r + a * a
    A = (r * r + a * a) ** 2 - a * a * Delta * s2
    return Sigma, Delta, A, s2


def fm_lnh(r, th, a, ell):
    """Unnormalised ln h of the torus (the integration constant is not removed)."""
    Sigma, Delta, A, s2 = _bl(r, th, a)
    e2nu = Sigma * Delta / A
    e2psi = A * s2 / Sigma
    omega = 2.0 * a * r / A
    s = np.sqrt(1.0 + 4.0 * ell * ell * e2nu / e2psi)
    return 0.5 * np.log((1.0 + s) / e2nu) - 0.5 * s - ell * omega


def fm_constants(a, r_in=6.0, r_pmax=12.0):
    """l with d(ln h)/dr = 0 at (r_pmax, pi/2), found by bisection on a
    central difference of ln h."""
    def slope(ell):
        h = 1e-4 * r_pmax
        return (fm_lnh(r_pmax + h, math.pi / 2, a, ell) - fm_lnh(r_pmax - h, math.pi / 2, a, ell)) / (2 * h)

    lo, hi = 1.0, 20.0
    assert slope(lo) * slope(hi) < 0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if slope(lo) * slope(mid) <= 0:
            hi = mid
        else:
            lo = mid
    ell = 0.5 * (lo + hi)
    lnh_in = float(fm_lnh(r_in, math.pi / 2, a, ell))
    return ell, lnh_in


def ks_code_metric(x1, x2, a):
    """Kerr-Schild lapse, radial shift and spatial metric in (ln r, th/pi, ph)."""
    r = np.exp(x1)
    th = np.pi * x2
    s2 = np.sin(th) ** 2
    Sigma = r * r + a * a * np.cos(th) ** 2
    z = 2.0 * r / Sigma
    g = np.zeros(np.shape(r) + (3, 3))
    g[..., 0, 0] = (1.0 + z) * r * r
    g[..., 0, 2] = g[..., 2, 0] = -a * s2 * (1.0 + z) * r
    g[..., 1, 1] = Sigma * np.pi * np.pi
    g[..., 2, 2] = s2 * (Sigma + a * a * s2 * (1.0 + z))
    alpha = 1.0 / np.sqrt(1.0 + z)
    beta1 = z / (1.0 + z) / r
    return alpha, beta1, g


def _torus_rho_p_uphi(r, th, a, gam, ell, lnh_in, K):
    """rho, p and the BL four-velocity (u^t, u^phi) inside the torus; rho = 0 outside."""
    with np.errstate(invalid="ignore", divide="ignore"):
        lnh = fm_lnh(r, th, a, ell) - lnh_in
    inside = np.isfinite(lnh) & (lnh > 0.0)
    h = np.exp(np.where(inside, lnh, 0.0))
    rho = np.where(inside, ((h - 1.0) * (gam - 1.0) / (K * gam)) ** (1.0 / (gam - 1.0)), 0.0)
    p = K * rho ** gam
    Sigma, Delta, A, s2 = _bl(r, th, a)
    e2nu = Sigma * Delta / A
    e2psi = A * s2 / Sigma
    omega = 2.0 * a * r / A
    with np.errstate(invalid="ignore", divide="ignore"):
        X = ell * np.sqrt(e2nu / e2psi)
        V = (-1.0 + np.sqrt(1.0 + 4.0 * X * X)) / (2.0 * X)
        gamma = 1.0 / np.sqrt(1.0 - V * V)
        ut = gamma / np.sqrt(e2nu)
        Om = omega + V * np.sqrt(e2nu / e2psi)
    uphi = Om * ut
    return inside, rho, p, ut, uphi


def fm_torus_prims(grid: Grid, r_in=6.0, r_pmax=12.0, beta=100.0, pert=0.02, seed=SEED,
                   field=True) -> np.ndarray:
    """Torus primitives on an MKS grid: FM equilibrium, rho_max = 1, a single
    poloidal loop A_phi = max(rho/rho_max - 0.2, 0) normalised to
    max p_gas / max p_mag = beta (p_mag = b^2/2), and a seeded uniform
    +-pert relative pressure perturbation in torus cells (rho > 10 rho_floor),
    drawn in cell order [block][k][j][i].  Outside: floor density and pressure
    at rest with respect to the normal observer."""
    assert grid.coords == "mks"
    if grid.ndim == 3 and grid.nx[2] > 1:
        # the equilibrium and the field do not depend on phi: build one plane
        # per block and repeat it, then draw the perturbation per cell
        flat = fm_torus_prims(grid.with_(nx=(grid.nx[0], grid.nx[1], 1)), r_in, r_pmax, beta, 0.0, seed, field)
        P = np.repeat(flat, grid.nx[2], axis=2)
        if pert > 0.0:
            _perturb(grid, P, pert, seed)
        return P
    a, gam = grid.spin, grid.gamma_ad
    ell, lnh_in = fm_constants(a, r_in, r_pmax)
    hmax = math.exp(float(fm_lnh(r_pmax, math.pi / 2, a, ell)) - lnh_in)
    K = (hmax - 1.0) * (gam - 1.0) / gam  # rho_max = 1
    x1, x2, x3 = cell_centres(grid)
    r, th = np.exp(x1), np.pi * x2
    inside, rho, p, ut, uphi = _torus_rho_p_uphi(r, th, a, gam, ell, lnh_in, K)
    inside &= r >= r_in
    alpha, beta1, g = ks_code_metric(x1, x2, a)
    P = empty_prims(grid)
    rho_fl = grid.rho_floor * r ** grid.rho_floor_pow
    p_fl = grid.p_floor * r ** grid.p_floor_pow
    P[:, 0] = np.where(inside, np.maximum(rho, rho_fl), rho_fl)
    P[:, 1] = np.where(inside, np.maximum(p, p_fl), p_fl)
    # code primitive u^i = W v^i = u^i(4-vel) + u^t beta^i; u^r = 0 in the torus
    P[:, 2] = np.where(inside, ut * beta1, 0.0)
    P[:, 4] = np.where(inside, uphi, 0.0)
    if field:
        B1, B2 = _loop_field(grid, a, gam, ell, lnh_in, K, r_in)
        # b^2 at cell centres with the code metric
        u = P[:, 2:5]
        B = np.stack([B1, B2, np.zeros_like(B1)], axis=1)
        ul = np.einsum("...ij,...j->...i", g, np.moveaxis(u, 1, -1))
        Bl = np.einsum("...ij,...j->...i", g, np.moveaxis(B, 1, -1))
        u2 = np.sum(np.moveaxis(u, 1, -1) * ul, axis=-1)
        W = np.sqrt(1.0 + u2)
        B2sq = np.sum(np.moveaxis(B, 1, -1) * Bl, axis=-1)
        Bv = np.sum(np.moveaxis(B, 1, -1) * ul, axis=-1) / W
        b2 = B2sq / (W * W) + Bv * Bv
        pmag_max = float(np.max(0.5 * b2))
        pgas_max = float(np.max(np.where(inside, P[:, 1], 0.0)))
        if pmag_max > 0.0:
            scale = math.sqrt(pgas_max / beta / pmag_max)
            P[:, 5] = B1 * scale
            P[:, 6] = B2 * scale
    if pert > 0.0:
        _perturb(grid, P, pert, seed)
    return P


def _perturb(grid, P, pert, seed):
    """p <- p (1 + pert (2 xi - 1)), xi ~ U[0, 1) in cell order, where rho > 10 rho_floor."""
    x1 = cell_centres(grid)[0]
    rho_fl = grid.rho_floor * np.exp(x1) ** grid.rho_floor_pow
    rng = np.random.default_rng(seed)
    xi = rng.random(P[:, 1].size).reshape(P[:, 1].shape)
    torus = P[:, 0] > 10.0 * rho_fl
    P[:, 1] = np.where(torus, P[:, 1] * (1.0 + pert * (2.0 * xi - 1.0)), P[:, 1])


def _loop_field(grid, a, gam, ell, lnh_in, K, r_in):
    """B^1, B^2 at cell centres from A_phi at the four cell corners in the
    (x1, x2) plane: B^1 = d_2 A_phi / sqrt(gamma), B^2 = -d_1 A_phi / sqrt(gamma)."""
    x1, x2, _ = cell_centres(grid)
    lev = grid.blocks[:, 0]
    dx1 = ((grid.xmax[0] - grid.xmin[0]) / (grid.nroot[0] * grid.nx[0] * 2.0 ** lev))[:, None, None, None]
    dx2 = ((grid.xmax[1] - grid.xmin[1]) / (grid.nroot[1] * grid.nx[1] * 2.0 ** lev))[:, None, None, None]

    def aphi(y1, y2):
        r, th = np.exp(y1), np.pi * y2
        inside, rho, _, _, _ = _torus_rho_p_uphi(r, th, a, gam, ell, lnh_in, K)
        rho = np.where(inside & (r >= r_in), rho, 0.0)
        return np.maximum(rho - 0.2, 0.0)

    amm = aphi(x1 - dx1 / 2, x2 - dx2 / 2)
    apm = aphi(x1 + dx1 / 2, x2 - dx2 / 2)
    amp = aphi(x1 - dx1 / 2, x2 + dx2 / 2)
    app = aphi(x1 + dx1 / 2, x2 + dx2 / 2)
    d1 = 0.5 * ((apm - amm) + (app - amp)) / dx1
    d2 = 0.5 * ((amp - amm) + (app - apm)) / dx2
    r, th = np.exp(x1), np.pi * x2
    Sigma = r * r + a * a * np.cos(th) ** 2
    z = 2.0 * r / Sigma
    sqrtg = Sigma * np.sin(th) * np.sqrt(1.0 + z) * r * np.pi
    return d2 / sqrtg, -d1 / sqrtg
