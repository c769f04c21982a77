"""Pins of the oracle's regridding with constrained transport (the face-field
transfer) against facts that do not come from the oracle:
- a divergence-free field linear in the coordinates is transferred exactly
  (refined faces, faces inside parent cells, coarsened faces);
- after refining a coarse block next to finer blocks that stay, and after
  coarsening, every cell's divergence is round-off, coarse faces on level
  boundaries are the mean of the finer ones, the copies of a face held by
  two blocks of one level are equal, the magnetic flux through every plane
  of the periodic box is unchanged, and so are the D, S_i, tau totals;
- refining a block and coarsening it again gives back its faces;
- the new grid keeps stepping with all of that intact.
CPU only."""
import numpy as np
import pytest

import oracle
import problems as pb
from problems import ct
from tests.test_oracle_ct_amr import _amr_field, _box, _copies_gap, _lattice

M3 = np.array([[0.3, 0.5, -0.2], [0.1, -0.7, 0.4], [0.6, -0.25, 0.4]])
B0 = np.array([1.1, -0.3, 0.45])


def _linear(g, d, X):
    """B = B0 + M x with trace M = 0 (2-D: the 2 x 2 block, M11 = -M00)."""
    M = M3.copy()
    if g.ndim == 2:
        M[2, :] = 0.0
        M[:, 2] = 0.0
        M[1, 1] = -M[0, 0]
    return B0[d] + sum(M[d, e] * X[e] for e in range(3))


def _faces_of(g, fn):
    return ct.join_faces(g, [np.broadcast_to(fn(g, d, _lattice(g, d, ring=False)), (g.nb,) + s)
                             for d, s in enumerate(ct.face_shapes(g))])


def _refine_root(g, root):
    """Leaves of g with level-0 block `root` split into its level-1 children."""
    nd = g.ndim
    out = [tuple(int(x) for x in b) for b in g.blocks if not (b[0] == 0 and tuple(b[1:1 + nd]) == root)]
    for s in range(1 << nd):
        c = [2 * root[e] + ((s >> e) & 1) for e in range(nd)] + [0] * (3 - nd)
        out.append((1, *c))
    return np.asarray(sorted(out), dtype=np.int32)


def _coarsen_root(g, root):
    nd = g.ndim
    out = [tuple(int(x) for x in b) for b in g.blocks
           if not (b[0] == 1 and tuple(int(x) >> 1 for x in b[1:1 + nd]) == root)]
    out.append((0, *root, *([0] * (3 - nd))))
    return np.asarray(sorted(out), dtype=np.int32)


def _root(ndim, i):
    return (i, 0) if ndim == 2 else (i, 0, 0)


@pytest.mark.parametrize("ndim", [2, 3])
def test_linear_field_is_transferred_exactly(ndim):
    """Outflow two-level box: refine the root block next to the refined one
    and coarsen the refined one in the same regrid; every new face equals the
    linear field at its centre."""
    g = _box(ndim, bc="outflow")
    o = oracle.Oracle(g)
    o.set_prims(pb.random_periodic_prims(g, jump=False))
    o.set_faces(_faces_of(g, _linear))
    g1 = g.with_(blocks=_coarsen_root(g.with_(blocks=_refine_root(g, _root(ndim, 1))), _root(ndim, 0)))
    o2 = o.regridded(g1.blocks)
    want = _faces_of(o2.grid, _linear)
    assert np.abs(o2.faces() - want).max() < 4e-15 * np.abs(want).max()


def _check(g, o, flux0, tot0, scale):
    F = o.faces()
    assert np.abs(ct.face_divergence(g, F)).max() < 1e-13 * scale
    assert ct.level_face_mismatch(g, F) < 1e-14 * scale
    assert _copies_gap(g, F) < 1e-14 * scale
    for d in range(g.ndim):
        assert np.allclose(ct.plane_fluxes(g, F, d), flux0[d], rtol=0, atol=1e-13), d
    vol = (0.5 ** g.ndim) ** g.blocks[:, 0].astype(float)
    U = o.cons()
    tot = np.array([(U[:, v].reshape(g.nb, -1).sum(axis=1) * vol).sum() for v in range(5)])
    assert np.abs(tot - tot0).max() < 1e-12 * np.abs(tot0).max(), tot - tot0


@pytest.mark.parametrize("ndim", [2, 3])
def test_regrids_keep_the_field_divergence_free_and_consistent(ndim):
    """Periodic two-level box with a random field and a mean field: refine the
    coarse root block beside the refined one (its new faces meet finer faces
    that stay), step, coarsen the first refined block, step.  (The random
    field is weak enough that no cell's pressure reaches its floor after a
    transfer: the totals are then exact.)"""
    g = _box(ndim)
    o = oracle.Oracle(g)
    o.set_prims(pb.random_periodic_prims(g, jump=False))
    F = _amr_field(g, amp=0.15)
    o.set_faces(F)
    scale = np.abs(F).max() * 32
    flux0 = [ct.plane_fluxes(g, F, d) for d in range(ndim)]
    vol = (0.5 ** ndim) ** g.blocks[:, 0].astype(float)
    U = o.cons()
    tot0 = np.array([(U[:, v].reshape(g.nb, -1).sum(axis=1) * vol).sum() for v in range(5)])
    g1 = g.with_(blocks=_refine_root(g, _root(ndim, 1)))
    o = o.regridded(g1.blocks)
    assert o.c2p_counts()[1:].sum() == 0
    _check(g1, o, flux0, tot0, scale)
    for _ in range(3):
        o.step(o.cfl_dt())
    U = o.cons()
    vol1 = (0.5 ** ndim) ** g1.blocks[:, 0].astype(float)
    tot1 = np.array([(U[:, v].reshape(g1.nb, -1).sum(axis=1) * vol1).sum() for v in range(5)])
    _check(g1, o, flux0, tot1, scale)
    assert np.abs(tot1 - tot0).max() < 1e-12 * np.abs(tot0).max()
    g2 = g1.with_(blocks=_coarsen_root(g1, _root(ndim, 0)))
    o = o.regridded(g2.blocks)
    _check(g2, o, flux0, tot1, scale)
    for _ in range(3):
        o.step(o.cfl_dt())
    assert o.c2p_counts()[1:].sum() == 0  # no floors: the totals are exact
    F2 = o.faces()
    assert np.abs(ct.face_divergence(g2, F2)).max() < 1e-13 * scale
    assert ct.level_face_mismatch(g2, F2) < 1e-14 * scale
    assert _copies_gap(g2, F2) < 1e-14 * scale


@pytest.mark.parametrize("ndim", [2, 3])
def test_refining_and_coarsening_again_restores_the_faces(ndim):
    g = _box(ndim)
    o = oracle.Oracle(g)
    o.set_prims(pb.random_periodic_prims(g, jump=False))
    F = _amr_field(g)
    o.set_faces(F)
    g1 = g.with_(blocks=_refine_root(g, _root(ndim, 1)))
    back = o.regridded(g1.blocks).regridded(g.blocks)
    assert np.abs(back.faces() - F).max() < 1e-14 * np.abs(F).max()


def test_three_level_torus_regrid_keeps_the_field_divergence_free():
    """The three-level torus (polar axis, phi + pi) regridded by its estimator's
    plan, refinement and coarsening together: every cell's divergence at
    round-off and the level boundaries consistent after the transfer and
    after a step."""
    g = pb.amr_torus(root=(4, 2, 2), nblock=8).with_(divb="ct")
    P = pb.fm_torus_prims(g)
    F = ct.fm_torus_faces(g, P)
    o = oracle.Oracle(g)
    o.set_prims(P)
    o.set_faces(F)
    new = o.regrid_plan(o.estimate(), 0.3, 0.05, 2)
    old_levels = {tuple(b) for b in np.asarray(g.blocks)}
    assert any(tuple(b) not in old_levels for b in new)
    o2 = o.regridded(new)
    g2 = o2.grid
    scale = np.abs(F).max() * 64
    for step in range(2):
        F2 = o2.faces()
        assert np.abs(ct.face_divergence(g2, F2)).max() < 1e-12 * scale, step
        assert ct.level_face_mismatch(g2, F2) < 1e-14 * scale, step
        assert np.all(np.isfinite(o2.cons()))
        o2.step(o2.cfl_dt())
