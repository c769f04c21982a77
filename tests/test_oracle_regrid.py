"""Pins of the oracle's AMR regridding against facts that do not come from
the oracle: Loehner's estimator in closed form on linear, step and quadratic
density profiles; leaf lists that tile the domain once, keep every pair of
touching leaves within one level (brute force over the finest-level cells,
periodic wrap and the polar axis included), refine every flagged block and
coarsen no block above the coarsening threshold; a conservative transfer
(volume integrals of every densitized conserved variable unchanged where no
floor acts), kept blocks copied bit for bit, and refinement followed by
coarsening returning the original state.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import problems as pb


def _box(ndim, nlevels=3, nroot=4, nblock=8):
    g = pb.periodic_box(ndim=ndim, nblock=nblock, nroot=nroot).with_(nlevels=nlevels, rho_floor=1e-30,
                                                                      p_floor=1e-30)
    return g


def _with_density(g, rho_fn):
    P = pb.empty_prims(g)
    xs = pb.cell_centres(g)
    P[:, 0] = rho_fn(*xs)
    P[:, 1] = 1.0
    return P


def test_estimator_closed_forms():
    g = _box(2, nlevels=1)
    eps = 0.01
    # linear density: zero second difference
    o = oracle.Oracle(g)
    o.set_prims(_with_density(g, lambda x, y, z: 1.0 + 0.3 * x + 0.2 * y))
    blk = np.asarray(g.blocks)
    inner = np.all((blk[:, 1:3] > 0) & (blk[:, 1:3] < 3), axis=1)  # away from the periodic seam
    assert inner.sum() == 4 and o.estimate(eps)[inner].max() < 1e-12
    # a step in x between two cells: at the cell left of it, 1-D value
    # 1 / (1 + 5 eps) combined with the y-direction filter term 4 eps
    o = oracle.Oracle(g)
    o.set_prims(_with_density(g, lambda x, y, z: np.where(x < 0.5, 1.0, 2.0)))
    e = o.estimate(eps)
    exact = 1.0 / math.sqrt((1 + 5 * eps) ** 2 + (4 * eps) ** 2)
    assert e.max() == pytest.approx(exact, rel=1e-14)
    # quadratic in x, far from the origin: N = 2 a h^2, D = 4 a |x| h + eps (4 rho),
    # checked cell by cell through the block maxima of a one-block-per-column grid
    a, x0 = 1.0, 2.0
    g1 = pb.Grid(ndim=2, nx=(8, 8, 1), nroot=(1, 1, 1), xmin=(x0, 0, 0), xmax=(x0 + 1, 1, 1), nlevels=1,
                 rho_floor=1e-30, p_floor=1e-30)
    o = oracle.Oracle(g1)
    o.set_prims(_with_density(g1, lambda x, y, z: a * x * x))
    h = 1.0 / 8
    xs = x0 + (np.arange(1, 7) + 0.5) * h  # interior cells whose neighbours are interior
    num = 2 * a * h * h
    den1 = np.abs(a * ((xs + h) ** 2 - xs ** 2)) + np.abs(a * (xs ** 2 - (xs - h) ** 2)) + eps * a * (
        (xs + h) ** 2 + 2 * xs ** 2 + (xs - h) ** 2)
    den2 = eps * 4 * a * xs ** 2
    est = num / np.sqrt(den1 ** 2 + den2 ** 2)
    # the block maximum is at least the largest interior value (the ghost-side
    # cells use outflow-free periodic wrap of a non-periodic profile, larger)
    assert o.estimate(eps)[0] >= est.max() * (1 - 1e-14)


def _finest_cells(grid, blocks, Lmax):
    """Cell boxes of each leaf at the finest level: (lo, hi) per dimension."""
    out = []
    for L, ix, iy, iz in blocks:
        f = 2 ** (Lmax - L)
        c = (ix, iy, iz)
        lo = [c[d] * grid.nx[d] * f if d < grid.ndim else 0 for d in range(3)]
        hi = [(c[d] + 1) * grid.nx[d] * f if d < grid.ndim else 1 for d in range(3)]
        out.append((lo, hi))
    return out


def _check_tiling_and_balance(grid, blocks, Lmax):
    N = [grid.nroot[d] * grid.nx[d] * 2 ** Lmax if d < grid.ndim else 1 for d in range(3)]
    owner = -np.ones(N[::-1], dtype=np.int64)
    boxes = _finest_cells(grid, blocks, Lmax)
    for n, (lo, hi) in enumerate(boxes):
        region = owner[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        assert np.all(region == -1), "leaves overlap"
        region[...] = n
    assert np.all(owner >= 0), "leaves do not tile the domain"
    levels = np.asarray(blocks)[:, 0]
    # neighbours: shift the owner map by one finest cell in every direction
    # (periodic where the boundary is, mirrored with phi + pi through an axis)
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in ((-1, 0, 1) if grid.ndim == 3 else (0,)):
                if dx == dy == dz == 0:
                    continue
                sh = np.roll(owner, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
                valid = np.ones(owner.shape, dtype=bool)
                for d, s in ((0, dx), (1, dy), (2, dz)):
                    if s == 0 or d >= grid.ndim:
                        continue
                    kind = grid.bc[d][0 if s < 0 else 1]
                    if kind == "periodic":
                        continue
                    ax = 2 - d
                    edge = [slice(None)] * 3
                    edge[ax] = 0 if s < 0 else owner.shape[ax] - 1
                    if kind == "axis":
                        # the mirrored neighbour of an axis row is the same row at phi + pi
                        mirrored = np.roll(owner, shift=owner.shape[0] // 2, axis=0) if grid.ndim == 3 else owner
                        sh[tuple(edge)] = mirrored[tuple(edge)]
                    else:
                        valid[tuple(edge)] = False
                diff = np.abs(levels[owner] - levels[sh])
                assert diff[valid].max() <= 1, "2:1 balance violated"


@pytest.mark.parametrize("ndim,seed", [(2, 1), (2, 39), (3, 3), (3, 5)])
def test_plan_tiles_the_domain_and_keeps_the_balance(ndim, seed):
    """Six successive plans on five levels with random (mostly small) errors:
    refinements, cascading balance and coarsening of whole sibling groups."""
    rng = np.random.default_rng(seed)
    g = _box(ndim, nlevels=5, nroot=3 if ndim == 3 else 4, nblock=4)
    blocks = np.asarray(g.blocks)
    for _ in range(6):
        o = oracle.Oracle(g.with_(blocks=blocks))
        err = rng.random(len(blocks)) ** 3
        new = o.regrid_plan(err, 0.5, 0.2, 4)
        _check_tiling_and_balance(g, new, 4)
        # every flagged block below the maximum level is refined
        newset = {tuple(b) for b in new}
        for b, e in zip(blocks, err):
            if e > 0.5 and b[0] < 4:
                assert tuple(b) not in newset
            if e >= 0.2:  # never coarsened: the block or its descendants remain
                parent = (b[0] - 1, b[1] // 2, b[2] // 2, b[3] // 2 if ndim == 3 else b[3])
                assert parent not in newset
        blocks = new
        if len(blocks) > 3000:
            break


def test_plan_balances_through_the_polar_axis():
    g = pb.amr_torus(root=(4, 2, 2), nblock=4)
    o = oracle.Oracle(g)
    rng = np.random.default_rng(9)
    err = rng.random(g.nb)
    new = o.regrid_plan(err, 0.7, 0.2, 2)
    _check_tiling_and_balance(g, new, 2)


def _random_state(g, seed=4):
    P = pb.random_periodic_prims(g, seed=seed)
    return P


def _totals(grid, cons):
    vol = 0.5 ** (grid.ndim * np.asarray(grid.blocks)[:, 0])
    return (cons * vol[:, None, None, None, None]).sum(axis=(0, 2, 3, 4))


@pytest.mark.parametrize("ndim", [2, 3])
def test_transfer_is_conservative_and_reversible(ndim):
    g = _box(ndim, nlevels=3, nroot=2, nblock=8)
    P = _random_state(g)
    o = oracle.Oracle(g)
    o.set_prims(P)
    rng = np.random.default_rng(11)
    err = rng.random(g.nb)
    fine = o.regrid_plan(err, 0.5, -1.0, 2)
    assert len(fine) > g.nb
    f = o.regridded(fine)
    assert np.all(f.c2p_counts()[2:] == 0)  # no floor or failure: the transfer alone
    t0, t1 = _totals(g, o.cons()), _totals(f.grid, f.cons())
    np.testing.assert_allclose(t1, t0, rtol=1e-13, atol=1e-13 * np.abs(t0).max())
    # kept blocks are copied bit for bit
    old = {tuple(b): n for n, b in enumerate(np.asarray(g.blocks))}
    for n, b in enumerate(np.asarray(fine)):
        if tuple(b) in old:
            assert np.array_equal(f.cons()[n], o.cons()[old[tuple(b)]])
    # coarsening everything back restores the original conserved state
    back = f.regrid_plan(np.zeros(len(fine)), 2.0, 1.0, 2)
    assert sorted(map(tuple, back)) == sorted(map(tuple, np.asarray(g.blocks)))
    r = f.regridded(back)
    order = [ {tuple(b): n for n, b in enumerate(back)}[tuple(b)] for b in np.asarray(g.blocks)]
    np.testing.assert_allclose(r.cons()[order], o.cons(), rtol=1e-14, atol=1e-14 * np.abs(o.cons()).max())


def test_regridded_grid_keeps_stepping():
    g = pb.amr_torus(root=(4, 2, 2), nblock=8)
    P = pb.fm_torus_prims(g)
    o = oracle.Oracle(g)
    o.set_prims(P)
    err = o.estimate()
    f = o.regridded(o.regrid_plan(err, 0.3, 0.05, 2))
    for _ in range(2):
        f.step(f.cfl_dt())
    assert np.all(np.isfinite(f.cons()))


def test_prolongation_is_exact_for_linear_fields():
    """At rest with no field in flat space, D = rho and tau = p/(Gamma - 1):
    linear density and pressure give linear conserved fields, which the
    minmod-limited prolongation reproduces exactly at the children's centres
    (away from the parent block's faces, where its slopes are one-sided and
    set to zero)."""
    g = _box(2, nlevels=2, nroot=2, nblock=8)
    P = _with_density(g, lambda x, y, z: 1.0 + 0.5 * x + 0.25 * y)
    P[:, 1] = 2.0 + 0.3 * pb.cell_centres(g)[0] - 0.2 * pb.cell_centres(g)[1]
    o = oracle.Oracle(g)
    o.set_prims(P)
    err = np.zeros(g.nb)
    err[0] = 1.0  # refine block 0 only
    f = o.regridded(o.regrid_plan(err, 0.5, -1.0, 1))
    fg = f.grid
    xs = pb.cell_centres(fg)
    fine = np.asarray(fg.blocks)[:, 0] == 1
    cons = f.cons()
    # children cells whose parent cell is not on the parent block's faces:
    # parent index 1..6 of 0..7 -> child global index 2..13 of 0..15
    gi = (np.asarray(fg.blocks)[:, 1, None] * 8 + np.arange(8)[None, :])
    gj = (np.asarray(fg.blocks)[:, 2, None] * 8 + np.arange(8)[None, :])
    ok_i = (gi >= 2) & (gi <= 13)
    ok_j = (gj >= 2) & (gj <= 13)
    mask = fine[:, None, None] & ok_j[:, :, None] & ok_i[:, None, :]
    D = cons[:, 0, 0]
    tau = cons[:, 4, 0]
    x, y = xs[0][:, 0], xs[1][:, 0]
    np.testing.assert_allclose(D[mask], (1.0 + 0.5 * x + 0.25 * y)[mask], rtol=1e-13)
    np.testing.assert_allclose(tau[mask], ((2.0 + 0.3 * x - 0.2 * y) / (5.0 / 3.0 - 1.0))[mask], rtol=1e-13)


def _flag(blocks, target):
    return np.array([1.0 if tuple(b) == target else 0.4 for b in np.asarray(blocks)])


def test_balance_cascades_across_levels():
    """Refining the corner block three times in a row: each new level forces
    its coarser neighbours, and theirs in turn, to refine (a chain of
    splits two levels deep), and every result keeps the 2:1 balance."""
    g = _box(2, nlevels=4, nroot=4, nblock=4)
    blocks = np.asarray(g.blocks)
    for L in range(3):
        o = oracle.Oracle(g.with_(blocks=blocks))
        target = (L, 2 ** L, 2 ** L, 0)  # the block at the centre-lower-left of the domain
        assert target in {tuple(b) for b in blocks}
        blocks = o.regrid_plan(_flag(blocks, target), 0.8, 0.1, 3)
        _check_tiling_and_balance(g, blocks, 3)
    assert np.bincount(np.asarray(blocks)[:, 0]).tolist()[3] == 4


def test_coarsening_that_would_break_the_balance_is_refused():
    """A level-2 group next to level-1 groups: asking every block to coarsen
    merges the level-2 group, but a level-1 group touching level-2 leaves may
    not become level 0 in the same pass."""
    g = _box(2, nlevels=3, nroot=4, nblock=4)
    blocks = np.asarray(g.blocks)
    blocks = oracle.Oracle(g.with_(blocks=blocks)).regrid_plan(_flag(blocks, (0, 1, 1, 0)), 0.8, 0.1, 2)
    blocks = oracle.Oracle(g.with_(blocks=blocks)).regrid_plan(_flag(blocks, (1, 2, 2, 0)), 0.8, 0.1, 2)
    levels = np.bincount(np.asarray(blocks)[:, 0], minlength=3)
    assert levels[2] == 4 and levels[1] > 4
    new = oracle.Oracle(g.with_(blocks=blocks)).regrid_plan(np.zeros(len(blocks)), 0.8, 0.5, 2)
    _check_tiling_and_balance(g, new, 2)
    lv = np.bincount(np.asarray(new)[:, 0], minlength=3)
    assert lv[2] == 0 and lv[1] > 0  # the level-2 group merged; its neighbours kept level 1
