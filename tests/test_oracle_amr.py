"""Pins of the oracle's cross-level ghost fill and coarse-fine flux correction
on a two-level block grid (CPU)."""
import math

import numpy as np
import pytest

import oracle
import problems as pb


def two_level_box(bc="periodic", n=8):
    """2x2 root blocks of n x n; root block (0, 0) refined into 4 level-1 blocks."""
    blocks = [(0, 1, 0, 0), (0, 0, 1, 0), (0, 1, 1, 0)] + [(1, i, j, 0) for j in (0, 1) for i in (0, 1)]
    g = pb.periodic_box(ndim=2, nblock=n, nroot=2).with_(
        nlevels=2, blocks=np.asarray(blocks, dtype=np.int32),
        bc=((bc, bc), (bc, bc), ("periodic", "periodic")))
    return g


def linear_prims(g, a=(1.0, 0.3, -0.2)):
    x, y, _ = pb.cell_centres(g)
    P = pb.empty_prims(g)
    for v in range(9):
        P[:, v] = (v + 1) * (a[0] + a[1] * x + a[2] * y) * (0.1 if v >= 2 else 1.0)
    return P


def ghost_values_expected(g, P, b, jj, ii):
    """Linear field value at the ghost cell's centre."""
    lev, bx, by, _ = g.blocks[b]
    n = g.nx[0]
    dx = 1.0 / (2 * n * 2 ** lev)
    x = (bx * n + ii - 3 + 0.5) * dx
    y = (by * n + jj - 3 + 0.5) * dx
    return x, y


def test_prolongation_and_restriction_exact_for_linear_data():
    """Linear data: minmod slopes are exact, so every interior ghost cell
    (away from the outflow boundary copies) equals the field at its centre,
    whether it is copied, prolongated from the coarse level or restricted from
    the fine level."""
    g = two_level_box("outflow")
    a = (1.0, 0.3, -0.2)
    P = linear_prims(g, a)
    o = oracle.Oracle(g)
    o.set_prims(P)
    o.fill_ghosts()
    G = o.prims_ghosted()
    checked = {"fine": 0, "coarse": 0}
    for b in range(g.nb):
        lev = g.blocks[b, 0]
        for jj in range(G.shape[3]):
            for ii in range(G.shape[4]):
                if 3 <= ii < 11 and 3 <= jj < 11:
                    continue
                x, y = ghost_values_expected(g, P, b, jj, ii)
                # skip cells whose stencil touches the domain edge (outflow copies)
                if not (0.25 / 8 * 3 < x < 1 - 0.25 / 8 * 3 and 0.25 / 8 * 3 < y < 1 - 0.25 / 8 * 3):
                    continue
                f = a[0] + a[1] * x + a[2] * y
                exp = np.array([(v + 1) * f * (0.1 if v >= 2 else 1.0) for v in range(9)])
                np.testing.assert_allclose(G[b, :, 0, jj, ii], exp, rtol=1e-13, atol=1e-14)
                checked["fine" if lev == 1 else "coarse"] += 1
    assert checked["fine"] > 50 and checked["coarse"] > 20


def test_restriction_of_fine_cells_is_their_mean():
    g = two_level_box("periodic")
    rng = np.random.default_rng(3)
    P = 1.0 + 0.1 * rng.random(size=(g.nb, 9, 1, 8, 8))
    o = oracle.Oracle(g)
    o.set_prims(P)
    o.fill_ghosts()
    G = o.prims_ghosted()
    # coarse block (1, 0) (index 0): its low-x ghosts at x in the refined region
    # are means of 2x2 fine cells of level-1 block (1, j)
    fine = {tuple(g.blocks[b, 1:3]): b for b in range(g.nb) if g.blocks[b, 0] == 1}
    for jj in range(3, 11):
        for ii in range(0, 3):
            jc = jj - 3           # coarse global j
            ic = 8 + ii - 3       # coarse global i (5..7)
            fi, fj = 2 * ic, 2 * jc
            vals = []
            for dj in (0, 1):
                for di in (0, 1):
                    I, J = fi + di, fj + dj
                    b = fine[(I // 8, J // 8)]
                    vals.append(P[b, :, 0, J % 8, I % 8])
            np.testing.assert_allclose(G[0, :, 0, jj, ii], np.mean(vals, axis=0), rtol=1e-15)


def test_two_level_conservation_with_reflux():
    """Periodic two-level box: the volume-weighted sums of D, S_i, tau, B^i are
    constant to round-off because coarse faces take the fine fluxes."""
    g = two_level_box("periodic")
    g = g.with_(kappa=0.5)
    P = pb.random_periodic_prims(g, jump=False)
    o = oracle.Oracle(g)
    o.set_prims(P)
    vol = np.array([1.0 / 4 ** lev for lev in g.blocks[:, 0]])[:, None, None, None]

    def totals():
        U = o.cons()
        return [math.fsum((U[:, v] * vol).ravel()) for v in range(8)], [
            math.fsum(np.abs(U[:, v] * vol).ravel()) for v in range(8)]

    t0, s0 = totals()
    for _ in range(20):
        o.step(o.cfl_dt())
    assert o.c2p_counts()[2:].sum() == 0
    t1, _ = totals()
    for v in range(8):
        assert abs(t1[v] - t0[v]) <= 1e-13 * s0[v], (v, t0[v], t1[v])
