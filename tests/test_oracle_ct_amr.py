"""Pins of the oracle's constrained transport across refinement levels against
facts that do not come from the oracle's own update:
- ring faces (the faces one cell outside a block) of a field that is linear
  along each face's normal and constant across it are the exact field values,
  whether they are copies, prolongations from a coarser leaf or restrictions
  of finer faces (the rule is exact for such a field);
- on two-level periodic boxes the discrete divergence of every cell stays at
  round-off, every coarse face on a level boundary stays the mean of the finer
  faces covering it, the copies of a face shared by two blocks of one level
  stay equal, the magnetic flux through every plane across the box is
  conserved, and so are the volume totals of D, S_i and tau;
- a field-free flow is evolved exactly as the pinned cleaning form evolves it
  on the same grid (the coarse-fine flux correction is the same);
- a circularly polarised Alfven wave through a refined patch has an error
  between those of the uniform coarse and uniform fine grids;
- the three-level torus keeps a divergence-free field through the axis.
CPU only."""
import math

import numpy as np
import pytest

import oracle
import problems as pb
from problems import ct
from tests.test_oracle_amr import two_level_box
from tests.test_oracle_ct import _alfven_setup


def two_level_box_3d(bc="periodic", n=8):
    """2x2x2 root blocks of n^3; root block (0, 0, 0) refined into 8 level-1 blocks."""
    blocks = [(0, i, j, k) for k in (0, 1) for j in (0, 1) for i in (0, 1) if (i, j, k) != (0, 0, 0)]
    blocks += [(1, i, j, k) for k in (0, 1) for j in (0, 1) for i in (0, 1)]
    return pb.periodic_box(ndim=3, nblock=n, nroot=2).with_(
        nlevels=2, blocks=np.asarray(blocks, dtype=np.int32), bc=((bc, bc),) * 3)


def _box(ndim, bc="periodic"):
    g = two_level_box(bc) if ndim == 2 else two_level_box_3d(bc)
    return g.with_(divb="ct")


def _lattice(grid, d, ring):
    """Coordinates of the faces normal to d of every block at its level:
    face-located along d (index 0..n_d), cell-centred across; with ring,
    across active directions the index runs -1..n_e."""
    out = []
    for e in range(3):
        lev = grid.blocks[:, 0].astype(np.int64)
        dx = (grid.xmax[e] - grid.xmin[e]) / (grid.nroot[e] * grid.nx[e]) / (2.0 ** lev if e < grid.ndim else np.ones(grid.nb))
        if e == d:
            idx, off = np.arange(grid.nx[e] + 1), 0.0
        elif ring and e < grid.ndim:
            idx, off = np.arange(-1, grid.nx[e] + 1), 0.5
        else:
            idx, off = np.arange(grid.nx[e]), 0.5
        x = grid.xmin[e] + (grid.blocks[:, 1 + e].astype(np.int64)[:, None] * grid.nx[e] + idx[None, :] + off) * dx[:, None]
        shape = [grid.nb, 1, 1, 1]
        shape[3 - e] = idx.size
        out.append(x.reshape(shape))
    return out


# Phi^d as a function of x_d only, divergence-free: sum of the slopes is zero
SLOPES = {2: (0.7, -0.7), 3: (0.7, -0.3, -0.4)}
OFFSETS = (1.3, -0.4, 0.25)


def _linear_field(grid, d, X):
    return OFFSETS[d] + SLOPES[grid.ndim][d] * X[d] + 0.0 * (X[0] + X[1] + X[2])


@pytest.mark.parametrize("ndim", [2, 3])
def test_ring_faces_are_exact_for_a_field_linear_along_the_normal(ndim):
    """Outflow two-level box: every ring face of every block (same-level
    copies, prolongations at even and odd positions along the normal,
    restrictions) equals the linear field at its position."""
    g = _box(ndim, bc="outflow")
    parts = [_linear_field(g, d, _lattice(g, d, ring=False)) for d in range(ndim)]
    F = ct.join_faces(g, [np.broadcast_to(p, (g.nb,) + s) for p, s in zip(parts, ct.face_shapes(g))])
    o = oracle.Oracle(g)
    o.set_prims(pb.random_periodic_prims(g, jump=False))
    o.set_faces(F)
    for d in range(ndim):
        ring = o.ring_faces(d)
        want = np.broadcast_to(_linear_field(g, d, _lattice(g, d, ring=True)), ring.shape)
        assert np.abs(ring - want).max() < 1e-14, (d, np.abs(ring - want).max())


def _amr_field(g, amp=0.3):
    """A smooth random divergence-free field plus a mean field (0.7, 0.4[, 0.3]),
    from a potential whose components do not depend on their own coordinate."""
    A1, A2, A3 = ct.own_potential_free(g, amp=amp)
    A3m = lambda x1, x2, x3: A3(x1, x2, x3) + 0.7 * x2 - 0.4 * x1
    if g.ndim == 2:
        return ct.faces_from_potential(g, A3=A3m)
    return ct.faces_from_potential(g, A1=A1, A2=lambda x1, x2, x3: A2(x1, x2, x3) + 0.3 * x1, A3=A3m)


def _copies_gap(g, F):
    """Largest difference between the copies of a face held by two blocks of
    the same level (periodic box)."""
    seen, worst = {}, 0.0
    for d, p in enumerate(ct.split_faces(g, F)):
        for b in range(g.nb):
            lev = int(g.blocks[b, 0])
            N = [g.nroot[e] * g.nx[e] * (2 ** lev if e < g.ndim else 1) for e in range(3)]
            k, j, i = np.meshgrid(*[np.arange(s) for s in p.shape[1:]], indexing="ij")
            G = [g.blocks[b, 1] * g.nx[0] + i, g.blocks[b, 2] * g.nx[1] + j, g.blocks[b, 3] * g.nx[2] + k]
            G[d] = G[d] % N[d]
            for key, v in zip(zip(G[0].ravel(), G[1].ravel(), G[2].ravel()), p[b].ravel()):
                key = (lev, d) + tuple(int(x) for x in key)
                if key in seen:
                    worst = max(worst, abs(seen[key] - v))
                else:
                    seen[key] = v
    return worst


@pytest.mark.parametrize("ndim, steps", [(2, 100), (3, 8)])
def test_two_level_box_keeps_the_field_divergence_free_and_consistent(ndim, steps):
    g = _box(ndim)
    P = pb.random_periodic_prims(g, jump=False)
    F = _amr_field(g)
    scale = np.abs(F).max() * 32
    assert np.abs(ct.face_divergence(g, F)).max() < 1e-14 * scale
    assert ct.level_face_mismatch(g, F) < 1e-15 * scale
    flux0 = [ct.plane_fluxes(g, F, d) for d in range(ndim)]
    o = oracle.Oracle(g)
    o.set_prims(P)
    o.set_faces(F)
    vol = (0.5 ** ndim) ** g.blocks[:, 0].astype(float)
    totals = lambda U: np.array([(U[:, v].reshape(g.nb, -1).sum(axis=1) * vol).sum() for v in range(5)])
    t0 = totals(o.cons())
    for _ in range(steps):
        o.step(o.cfl_dt())
    F2 = o.faces()
    assert o.c2p_counts()[1:].sum() == 0  # no floors, no backup: the totals are exact
    assert np.abs(F2 - F).max() > 0.1 * np.abs(F).max()
    assert np.abs(ct.face_divergence(g, F2)).max() < 1e-13 * scale
    assert ct.level_face_mismatch(g, F2) < 1e-14 * scale
    assert _copies_gap(g, F2) < 1e-14 * scale
    for d in range(ndim):
        assert np.allclose(ct.plane_fluxes(g, F2, d), flux0[d], rtol=0, atol=1e-13), d
    t1 = totals(o.cons())
    assert np.abs(t1 - t0).max() < 1e-12 * np.abs(t0).max(), (t1 - t0)


@pytest.mark.parametrize("ndim", [2, 3])
def test_field_free_flow_matches_the_cleaning_form_across_levels(ndim):
    """B = 0 on a two-level box: constrained transport and the cleaning form
    evolve D, S_i, tau with the same fluxes and the same coarse-fine
    correction, so equal steps give bit-identical hydrodynamics."""
    g0 = _box(ndim).with_(divb="glm")
    P = pb.random_periodic_prims(g0)
    P[:, 5:9] = 0.0
    og = oracle.Oracle(g0)
    og.set_prims(P)
    oc = oracle.Oracle(g0.with_(divb="ct"))
    oc.set_prims(P)
    oc.set_faces(np.zeros(ct.face_count(g0)))
    dt = 0.5 * og.cfl_dt()
    for _ in range(3 if ndim == 2 else 1):
        og.step(dt)
        oc.step(dt)
    assert np.array_equal(og.cons()[:, :5], oc.cons()[:, :5])


def _alfven_error(g, t_end=0.25):
    P0, F0, _ = _alfven_setup(g, 0, 0.0)
    o = oracle.Oracle(g)
    o.set_prims(P0)
    o.set_faces(F0)
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(o.cfl_dt(), t_end - t)
        o.step(dt)
        t += dt
    Pe, _, _ = _alfven_setup(g, 0, t_end)
    vol = 0.25 ** g.blocks[:, 0].astype(float)
    err = np.abs(o.prims()[:, 6] - Pe[:, 6]).reshape(g.nb, -1).mean(axis=1)
    return float((err * vol).sum() / vol.sum()), o


def test_alfven_wave_through_a_refined_patch():
    """The wave along x crosses a refined root block (level boundaries normal
    to x and to y): its L1 error lies between the uniform fine grid's and 1.15
    times the uniform coarse grid's (the cleaning form's AMR error on the same
    grids is 1.10 times its coarse error), and the field stays
    divergence-free and consistent across the levels."""
    base = pb.Grid(ndim=2, nx=(8, 8, 1), nroot=(4, 2, 1), xmin=(0, 0, 0), xmax=(1, 0.5, 1), gamma_ad=5.0 / 3.0,
                   recon="ppm", riemann="hll", cfl=0.4, divb="ct")
    fine = base.with_(nroot=(8, 4, 1), blocks=pb.uniform_blocks((8, 4, 1)))
    blocks = [(0, i, j, 0) for j in range(2) for i in range(4) if (i, j) != (1, 0)]
    blocks += [(1, i, j, 0) for j in (0, 1) for i in (2, 3)]
    amr = base.with_(nlevels=2, blocks=np.asarray(blocks, dtype=np.int32))
    e_coarse, _ = _alfven_error(base)
    e_fine, _ = _alfven_error(fine)
    e_amr, o = _alfven_error(amr)
    assert e_fine < e_amr < 1.15 * e_coarse, (e_fine, e_amr, e_coarse)
    F = o.faces()
    scale = np.abs(F).max() * 32
    assert np.abs(ct.face_divergence(amr, F)).max() < 1e-13 * scale
    assert ct.level_face_mismatch(amr, F) < 1e-14 * scale


def test_three_level_torus_keeps_the_field_divergence_free():
    """Modified Kerr-Schild torus on three levels with the loop field as faces
    (its potential A_phi does not depend on phi, so the levels start
    consistent): after three steps every cell's divergence is round-off, the
    level boundaries stay consistent and the axis faces carry no field."""
    g = pb.amr_torus(root=(4, 2, 2), nblock=8).with_(divb="ct")
    P = pb.fm_torus_prims(g)
    F = ct.fm_torus_faces(g, P)
    scale = np.abs(F).max() * 64
    assert ct.level_face_mismatch(g, F) < 1e-15 * scale
    o = oracle.Oracle(g)
    o.set_prims(P)
    o.set_faces(F)
    for _ in range(3):
        o.step(o.cfl_dt())
    F2 = o.faces()
    assert np.all(np.isfinite(o.cons()))
    assert np.abs(F2 - F).max() > 0.0
    assert np.abs(ct.face_divergence(g, F2)).max() < 1e-12 * scale
    assert ct.level_face_mismatch(g, F2) < 1e-14 * scale
    p2 = ct.split_faces(g, F2)[1]
    top = g.nroot[1] * 2 ** g.blocks[:, 0] - 1
    assert np.all(p2[g.blocks[:, 2] == 0][:, :, 0, :] == 0.0)
    assert np.all(p2[g.blocks[:, 2] == top][:, :, -1, :] == 0.0)


@pytest.mark.parametrize("ndim, divb", [(2, "ct"), (3, "ct"), (2, "glm"), (3, "glm")])
def test_grid_entirely_at_level_one_is_the_uniform_finer_grid(ndim, divb):
    """Every leaf at level 1 of a two-level description is the uniform grid
    with twice the root blocks: the level-aware paths (spacings, global
    indices, ring faces and boundary rules at the leaves' level, the EMFs)
    must reproduce the uniform run bit for bit."""
    n = 8
    fine = pb.periodic_box(ndim=ndim, nblock=n, nroot=4).with_(divb=divb)
    if ndim == 2:
        blocks = [(1, i, j, 0) for j in range(4) for i in range(4)]
    else:
        blocks = [(1, i, j, k) for k in range(4) for j in range(4) for i in range(4)]
    lev = pb.periodic_box(ndim=ndim, nblock=n, nroot=2).with_(
        divb=divb, nlevels=2, blocks=np.asarray(blocks, dtype=np.int32))
    # the same leaves in the same order, so the arrays line up block by block
    assert np.array_equal(np.asarray(lev.blocks)[:, 1:], np.asarray(fine.blocks)[:, 1:])
    P = pb.random_periodic_prims(fine, jump=False)
    outs = []
    for g in (fine, lev):
        o = oracle.Oracle(g)
        o.set_prims(P)
        if divb == "ct":
            o.set_faces(ct.random_potential_faces(fine))
        for _ in range(3 if ndim == 2 else 1):
            o.step(o.cfl_dt())
        outs.append((o.cons(), o.faces() if divb == "ct" else None))
    assert np.array_equal(outs[0][0], outs[1][0])
    if divb == "ct":
        assert np.array_equal(outs[0][1], outs[1][1])
