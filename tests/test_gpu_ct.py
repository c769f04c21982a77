"""Constrained transport on the GPU against the FP64 oracle, through the C ABI.

Face fields Phi^d = sqrt(gamma) B^d and the conserved state after one and
several steps from the same seeded input: conserved variables within 1e-12
(energy-scaled, as in test_gpu_parity), face fields within 1e-12 of the
largest face field; the GPU's faces keep every cell's discrete divergence at
round-off.  Grids: periodic boxes in 2-D and 3-D with a random divergence-free
field, the shock tube, and the torus in modified Kerr-Schild coordinates with
the polar axis (2-D and 3-D); across refinement levels two-level periodic
boxes (2-D, 3-D) and the three-level torus, where the coarse faces on level
boundaries also stay the mean of the finer faces covering them."""
import numpy as np
import pytest

import oracle
import problems as pb
from problems import ct

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_2108_12240_gb300 as m
    return m


def _case(name):
    if name == "box2d":
        g = pb.periodic_box(ndim=2, nblock=16, nroot=3).with_(divb="ct")
        return g, pb.random_periodic_prims(g, jump=True), None
    if name == "box3d":
        g = pb.periodic_box(ndim=3, nblock=8, nroot=2).with_(divb="ct")
        return g, pb.random_periodic_prims(g, jump=True), None
    if name == "shock_tube":
        g = pb.shock_tube_2d().with_(divb="ct")
        return g, pb.shock_tube_prims(g), ct.shock_tube_faces(g)
    if name == "torus2d":
        g = pb.torus_2d(nblock=16, nroot=(6, 4)).with_(divb="ct")
        P = pb.fm_torus_prims(g)
        return g, P, ct.fm_torus_faces(g, P)
    if name in ("amr_box2d", "amr_box3d"):
        from tests.test_oracle_ct_amr import _amr_field, _box
        g = _box(2 if name == "amr_box2d" else 3)
        return g, pb.random_periodic_prims(g, jump=True), _amr_field(g)
    if name == "amr_torus":
        g = pb.amr_torus(root=(4, 2, 2), nblock=8).with_(divb="ct")
        P = pb.fm_torus_prims(g)
        return g, P, ct.fm_torus_faces(g, P)
    g = pb.torus_3d(nroot=(4, 3, 2)).with_(divb="ct")
    P = pb.fm_torus_prims(g)
    return g, P, ct.fm_torus_faces(g, P)


def _faces(g, F):
    return ct.random_potential_faces(g) if F is None else F


def _dxmin(g):
    """The finest cell width of the grid."""
    return min((g.xmax[d] - g.xmin[d]) / (g.nroot[d] * g.nx[d]) for d in range(g.ndim)) / 2 ** (g.nlevels - 1)


@pytest.mark.parametrize("name", ["box2d", "box3d", "shock_tube", "torus2d", "torus3d", "amr_box2d", "amr_box3d",
                                  "amr_torus"])
def test_ct_matches_oracle(gb, name):
    from tests.test_gpu_parity import energy_scaled
    g, P, F = _case(name)
    F = _faces(g, F)
    s = gb.Solver(g)
    s.set_prims(P)
    s.set_faces(F)
    o = oracle.Oracle(g)
    o.set_prims(P)
    o.set_faces(F)
    # the loaded state: cell field from the faces, same conserved variables
    assert np.abs(s.cons() - o.cons()).max() <= 1e-14 * np.abs(o.cons()).max()
    for step in range(3):
        dt = o.cfl_dt()
        assert s.cfl_dt() == pytest.approx(dt, rel=1e-13)
        o.step(dt)
        s.step(dt)
        got, ref = s.cons(), o.cons()
        assert np.all(np.isfinite(got))
        err = energy_scaled(got, ref, g)
        assert np.all(err <= TOL64), (step, err)
        fg, fo = s.faces(), o.faces()
        scale = np.abs(fo).max()
        assert np.abs(fg - fo).max() <= TOL64 * scale, (step, np.abs(fg - fo).max() / scale)
        div = np.abs(ct.face_divergence(g, fg)).max()
        assert div <= 1e-12 * scale / _dxmin(g), div
        if g.nlevels > 1:
            assert ct.level_face_mismatch(g, fg) <= 1e-13 * scale
    print(f"CT {name}: energy-scaled error per conserved variable after 3 steps {err.tolist()}")


@pytest.mark.parametrize("name", ["torus2d", "amr_torus"])
def test_ct_device_dt_and_graph_replay_are_bitwise_identical(gb, name):
    """Steps with the device time step, direct and replayed from a CUDA graph,
    give the same bits; the face buffers' roles return after every step."""
    g, P, F = _case(name)
    outs = []
    for mode in ("direct", "graph"):
        import torch
        st = torch.cuda.Stream()
        s = gb.Solver(g, stream=st)
        s.set_prims(P)
        s.set_faces(F)
        s.cfl_dt()
        if mode == "direct":
            for _ in range(4):
                s.step(0.0)
        else:
            s.capture(2)
            s.replay()
            s.replay()
        st.synchronize()
        outs.append((s.cons(), s.faces()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("name", ["box3d", "amr_box3d"])
def test_ct_keeps_the_divergence_at_round_off_over_many_steps(gb, name):
    g, P, F = _case(name)
    F = _faces(g, F)
    s = gb.Solver(g)
    s.set_prims(P)
    s.set_faces(F)
    s.cfl_dt()
    for _ in range(60):
        s.step(0.0)
    fg = s.faces()
    assert np.abs(fg - F).max() > 0.1 * np.abs(F).max()
    assert np.abs(ct.face_divergence(g, fg)).max() <= 1e-12 * np.abs(fg).max() / _dxmin(g)
    assert np.all(s.prims()[:, 8] == 0.0)
    if g.nlevels > 1:
        assert ct.level_face_mismatch(g, fg) <= 1e-13 * np.abs(fg).max()
        for d in range(g.ndim):
            assert np.allclose(ct.plane_fluxes(g, fg, d), ct.plane_fluxes(g, F, d), rtol=0, atol=1e-12)


def test_ct_call_order_and_forms(gb):
    """A step before the faces are loaded, and face calls on a cleaning-form
    grid, are call-order errors."""
    g, P, F = _case("box2d")
    s = gb.Solver(g)
    s.set_prims(P)
    with pytest.raises(gb.BhacError) as e:
        s.step(1e-3)
    assert e.value.status == 4
    glm = gb.Solver(g.with_(divb="glm"))
    glm.set_prims(P)
    with pytest.raises(gb.BhacError) as e:
        glm.set_faces(ct.random_potential_faces(g))
    assert e.value.status == 4


@pytest.mark.parametrize("name", ["box2d", "box3d", "torus2d", "torus3d", "amr_box3d", "amr_torus"])
def test_ct_mixed_form_matches_oracle(gb, name):
    """The mixed form of constrained transport (FP32 face states and fluxes,
    FP64 EMFs, face update and face field) against the FP64 oracle: after one
    step, conserved variables within the mixed form's per-step bar of 1e-5
    (energy-scaled) and face fields within 1e-5 of the largest one; after two
    more, every cell's discrete divergence still at FP64 round-off."""
    from tests.test_gpu_parity import energy_scaled
    g, P, F = _case(name)
    F = _faces(g, F)
    s = gb.Solver(g, "mixed")
    s.set_prims(P)
    s.set_faces(F)
    o = oracle.Oracle(g)
    o.set_prims(P)
    o.set_faces(F)
    dt = o.cfl_dt()
    o.step(dt)
    s.step(dt)
    err = energy_scaled(s.cons(), o.cons(), g)
    assert np.all(err <= 1e-5), err
    fg, fo = s.faces(), o.faces()
    scale = np.abs(fo).max()
    assert np.abs(fg - fo).max() <= 1e-5 * scale
    for _ in range(2):
        s.step(0.0)
    fg = s.faces()
    assert np.abs(ct.face_divergence(g, fg)).max() <= 1e-12 * np.abs(fg).max() / _dxmin(g)
    if g.nlevels > 1:
        assert ct.level_face_mismatch(g, fg) <= 1e-13 * np.abs(fg).max()
    print(f"CT mixed {name}: energy-scaled error per conserved variable after a step {err.tolist()}")


@pytest.mark.parametrize("name, variant", [("amr_box2d", dict(recon="minmod", riemann="tvdlf")),
                                           ("amr_box3d", dict(recon="minmod")),
                                           ("amr_torus", dict(riemann="tvdlf")),
                                           ("amr_torus", dict(c2p="nk"))])
def test_ct_across_levels_scheme_variants(gb, name, variant):
    """Constrained transport across levels with the other reconstruction and
    Riemann solver, and with the Newton-Krylov inversion: two steps at the
    oracle's time step, conserved variables within 1e-12 (energy-scaled),
    faces within 1e-12 of the largest, divergence and level boundaries at
    round-off."""
    from tests.test_gpu_parity import energy_scaled
    g, P, F = _case(name)
    g = g.with_(**variant)
    F = _faces(g, F)
    s = gb.Solver(g)
    s.set_prims(P)
    s.set_faces(F)
    o = oracle.Oracle(g)
    o.set_prims(P)
    o.set_faces(F)
    for _ in range(2):
        dt = o.cfl_dt()
        o.step(dt)
        s.step(dt)
    err = energy_scaled(s.cons(), o.cons(), g)
    assert np.all(err <= TOL64), err
    fg, fo = s.faces(), o.faces()
    scale = np.abs(fo).max()
    assert np.abs(fg - fo).max() <= TOL64 * scale
    assert np.abs(ct.face_divergence(g, fg)).max() <= 1e-12 * scale / _dxmin(g)
    assert ct.level_face_mismatch(g, fg) <= 1e-13 * scale


@pytest.mark.parametrize("ndim, divb, form", [(2, "ct", "fp64"), (3, "ct", "fp64"), (3, "ct", "mixed"),
                                              (3, "glm", "fp64")])
def test_grid_entirely_at_level_one_is_the_uniform_finer_grid(gb, ndim, divb, form):
    """The library's level paths (per-level spacings and tables, the level
    maps of constrained transport with nothing to correct) on a grid whose
    leaves are all at level 1 give the uniform finer grid's result (the
    1/dx of level 1 is the uniform grid's exactly on this unit box)."""
    n = 8
    fine = pb.periodic_box(ndim=ndim, nblock=n, nroot=4).with_(divb=divb)
    blocks = [(1, i, j, k) for k in range(4 if ndim == 3 else 1) for j in range(4) for i in range(4)]
    lev = pb.periodic_box(ndim=ndim, nblock=n, nroot=2).with_(
        divb=divb, nlevels=2, blocks=np.asarray(blocks, dtype=np.int32))
    P = pb.random_periodic_prims(fine, jump=False)
    outs = []
    for g in (fine, lev):
        s = gb.Solver(g, form)
        s.set_prims(P)
        if divb == "ct":
            s.set_faces(ct.random_potential_faces(fine))
        s.cfl_dt()
        for _ in range(3):
            s.step(0.0)
        outs.append((s.cons(), s.faces() if divb == "ct" else None))
    scale = np.abs(outs[0][0]).max()
    assert np.abs(outs[0][0] - outs[1][0]).max() <= 1e-14 * scale
    if divb == "ct":
        assert np.abs(outs[0][1] - outs[1][1]).max() <= 1e-14 * np.abs(outs[0][1]).max()
