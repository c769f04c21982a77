"""Pins of the oracle's staggered-mesh constrained transport against facts
that do not come from the oracle: the discrete divergence of every cell stays
at round-off, the field's volume integral is conserved in a periodic box, a
field-free flow is evolved exactly as the pinned cleaning form evolves it,
and circularly polarised Alfven waves along each axis (closed-form travelling
solutions) converge at second order.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import problems as pb
from problems import ct


def _run(grid, P, F, steps, dt=None):
    o = oracle.Oracle(grid)
    o.set_prims(P)
    o.set_faces(F)
    for _ in range(steps):
        o.step(dt if dt is not None else o.cfl_dt())
    return o


@pytest.mark.parametrize("ndim", [2, 3])
def test_ct_keeps_the_discrete_divergence_at_round_off(ndim):
    """Random smooth state and random divergence-free field in a periodic box:
    after many steps every cell's sum_d dPhi^d/dx_d is still round-off of
    |Phi|/dx, the field changed at order one, psi stays exactly zero, and the
    sums of the face fields over each direction (the box's mean field) are
    conserved."""
    g = pb.periodic_box(ndim=ndim, nblock=8, nroot=2).with_(divb="ct")
    P = pb.random_periodic_prims(g, jump=False)
    F = ct.random_potential_faces(g)
    scale = np.abs(F).max() * 16
    assert np.abs(ct.face_divergence(g, F)).max() < 1e-14 * scale
    o = _run(g, P, F, 30 if ndim == 2 else 8)
    F2 = o.faces()
    assert np.abs(F2 - F).max() > 0.1 * np.abs(F).max()
    assert np.abs(ct.face_divergence(g, F2)).max() < 1e-13 * scale
    assert np.all(o.prims()[:, 8] == 0.0)
    for d, (p0, p1) in enumerate(zip(ct.split_faces(g, F), ct.split_faces(g, F2))):
        # each block's faces 0..nx_d - 1 along d tile the periodic box once
        ax = 3 - d
        lo0 = p0.take(range(p0.shape[ax] - 1), axis=ax)
        lo1 = p1.take(range(p1.shape[ax] - 1), axis=ax)
        assert np.sum(lo1) == pytest.approx(np.sum(lo0), rel=1e-12, abs=1e-13 * np.abs(lo0).sum())


def test_ct_torus_keeps_divergence_free_through_the_axis():
    """The Fishbone-Moncrief torus with its loop field as faces, modified
    Kerr-Schild, polar axis at both x2 boundaries: div B stays at round-off
    and the state stays finite."""
    g = pb.torus_2d(nblock=8, nroot=(4, 4)).with_(divb="ct")
    P = pb.fm_torus_prims(g)
    F = ct.fm_torus_faces(g, P)
    parts = ct.split_faces(g, F)
    scale = max(np.abs(p).max() for p in parts) * 32
    o = _run(g, P, F, 5)
    F2 = o.faces()
    assert np.all(np.isfinite(o.cons()))
    assert np.abs(F2 - F).max() > 0.0
    assert np.abs(ct.face_divergence(g, F2)).max() < 1e-12 * scale
    # the axis faces carry no field
    p2 = ct.split_faces(g, F2)[1]
    blocks = np.asarray(g.blocks)
    assert np.all(p2[blocks[:, 2] == 0][:, :, 0, :] == 0.0)
    assert np.all(p2[blocks[:, 2] == g.nroot[1] - 1][:, :, -1, :] == 0.0)


def test_ct_without_field_matches_the_cleaning_form():
    """B = 0: the constrained-transport and cleaning forms evolve D, S_i, tau
    with the same operations (no field flux, no cleaning), so equal steps give
    bit-identical hydrodynamics."""
    g0 = pb.periodic_box(ndim=2, nblock=8, nroot=2)
    P = pb.random_periodic_prims(g0)
    P[:, 5:9] = 0.0
    og = oracle.Oracle(g0)
    og.set_prims(P)
    oc = oracle.Oracle(g0.with_(divb="ct"))
    oc.set_prims(P)
    oc.set_faces(np.zeros(ct.face_count(g0)))
    dt = 0.5 * og.cfl_dt()
    for _ in range(5):
        og.step(dt)
        oc.step(dt)
    assert np.array_equal(og.cons()[:, :5], oc.cons()[:, :5])


def _alfven_setup(grid, axis, t, b0=1.0, eta=1.0, rho=1.0, p=1.0):
    """Circularly polarised Alfven wave travelling along `axis` (0, 1, 2):
    the closed form of problems.alfven_wave_prims with the axes permuted.
    Returns primitives and faces from the vector potential
    A_{a2} = b0 x_{a1} - eta b0 sin(k s)/k, A_{a1} = -eta b0 cos(k s)/k
    (s = x_axis - vA t; (axis, a1, a2) cyclic), whose curl is the wave's field."""
    xs = pb.cell_centres(grid)
    k = 2.0 * math.pi
    vA = pb.alfven_speed(rho, p, grid.gamma_ad, b0, eta)
    s = xs[axis] - vA * t
    a1, a2 = (axis + 1) % 3, (axis + 2) % 3
    Bt1, Bt2 = eta * b0 * np.cos(k * s), eta * b0 * np.sin(k * s)
    v1, v2 = -vA * Bt1 / b0, -vA * Bt2 / b0
    W = 1.0 / np.sqrt(1.0 - v1 * v1 - v2 * v2)
    P = pb.empty_prims(grid)
    P[:, 0] = rho
    P[:, 1] = p
    P[:, 2 + a1] = W * v1
    P[:, 2 + a2] = W * v2
    P[:, 5 + axis] = b0
    P[:, 5 + a1] = Bt1
    P[:, 5 + a2] = Bt2
    # vector potential: B_axis = b0 from A_{a2} = b0 x_{a1} (curl), the transverse
    # components from A_{a1}, A_{a2} functions of x_axis only
    A = [None, None, None]
    xa = lambda X: X[axis] - vA * t
    A[a2] = lambda *X: b0 * X[a1] - eta * b0 * np.sin(k * xa(X)) / k
    A[a1] = lambda *X: -eta * b0 * np.cos(k * xa(X)) / k
    # (in 2-D with the wave along x only A_3 enters the faces; B^3 is a cell value)
    F = ct.faces_from_potential(grid, A1=A[0], A2=A[1], A3=A[2])
    return P, F, vA


def _alfven_l1(n, axis, ndim):
    cells = [4, 4, 4]
    cells[axis] = n
    nx = tuple(min(c, 16) if d < ndim else 1 for d, c in enumerate(cells))
    nroot = tuple(cells[d] // nx[d] if d < ndim else 1 for d in range(3))
    xmax = tuple(cells[d] / n if d < ndim else 1.0 for d in range(3))
    g = pb.Grid(ndim=ndim, nx=nx, nroot=nroot, xmin=(0, 0, 0), xmax=xmax, gamma_ad=5.0 / 3.0,
                recon="ppm", riemann="hll", cfl=0.4, divb="ct")
    P0, F0, _ = _alfven_setup(g, axis, 0.0)
    o = oracle.Oracle(g)
    o.set_prims(P0)
    o.set_faces(F0)
    t, t_end = 0.0, 0.25
    while t < t_end - 1e-14:
        dt = min(o.cfl_dt(), t_end - t)
        o.step(dt)
        t += dt
    Pe, _, _ = _alfven_setup(g, axis, t_end)
    a1 = (axis + 1) % 3
    return float(np.mean(np.abs(o.prims()[:, 5 + a1] - Pe[:, 5 + a1])))


@pytest.mark.parametrize("ndim,axis", [(2, 0), (3, 1), (3, 2)])
def test_ct_alfven_wave_converges_at_second_order(ndim, axis):
    """Errors at t = 0.25 fall at order >= 1.8 from 16 to 32 to 64 cells along
    the wave: the EMF averaging and the curl update carry the induction
    equation (in 3-D along y and z every EMF component takes part)."""
    e = [_alfven_l1(n, axis, ndim) for n in (16, 32, 64)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(orders) > 1.8, (e, orders)
