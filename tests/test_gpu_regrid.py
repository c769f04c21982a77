"""AMR regridding on the GPU against the FP64 oracle, through the C ABI:
the per-block estimator (1e-12 relative), the transferred state (conserved
variables within 1e-12 energy-scaled in the FP64 form, 1e-5 in the mixed
form; per-cell inversion outcome equal) and one step on the new grid; with
constrained transport also the transferred face fields.  The plan itself is
host code, compared with the oracle's in test_regrid_plan_host."""
import numpy as np
import pytest

import oracle
import problems as pb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_2108_12240_gb300 as m
    return m


def _case(name):
    if name == "amr_torus":
        g = pb.amr_torus(root=(4, 2, 2), nblock=8)
        return g, pb.fm_torus_prims(g), (0.3, 0.05, 2)
    g = pb.periodic_box(ndim=3, nblock=8, nroot=2).with_(nlevels=3, rho_floor=1e-30, p_floor=1e-30)
    return g, pb.random_periodic_prims(g), (0.5, 0.1, 2)


@pytest.mark.parametrize("name,form,tol", [("amr_torus", "fp64", 1e-12), ("box3d", "fp64", 1e-12),
                                           ("amr_torus", "mixed", 1e-5)])
def test_regrid_matches_oracle(gb, name, form, tol):
    from tests.test_gpu_parity import energy_scaled
    g, P, (tr, tc, maxl) = _case(name)
    s = gb.Solver(g, form)
    s.set_prims(P)
    o = oracle.Oracle(g)
    o.set_prims(P)
    if name == "box3d":  # a refined box first, so the regrid below both refines and coarsens
        e0 = np.linspace(0.0, 1.0, g.nb)
        b1 = o.regrid_plan(e0, 0.5, -1.0, maxl)
        o = o.regridded(b1)
        s = s.regridded(b1)
        g = o.grid
    err_o = o.estimate()
    err_s = s.estimate()
    if form == "fp64":
        np.testing.assert_allclose(err_s, err_o, rtol=1e-12, atol=1e-15)
    else:
        np.testing.assert_allclose(err_s, err_o, rtol=1e-4, atol=1e-6)
    new = o.regrid_plan(err_o, tr, tc, maxl)
    assert not np.array_equal(new, np.asarray(g.blocks))
    on = o.regridded(new)
    sn = s.regridded(new)
    got, ref = sn.cons(), on.cons()
    assert np.all(np.isfinite(got))
    err = energy_scaled(got, ref, on.grid)
    assert np.all(err <= tol), ("transfer", err)
    if form == "fp64":
        # the transferred atmosphere holds its pressure at the floor, and the
        # inversion recovers that pressure from a cancellation in tau with a
        # relative error near 1e-11: whether the floor then applies is decided
        # by rounding, so such cells may swap between "converged" and
        # "floored" (the state agrees either way, checked above); no other
        # outcome may differ
        gs, os_ = sn.c2p_status(), on.c2p_status()
        diff = gs != os_
        pairs = {(int(x), int(y)) for x, y in zip(gs[diff], os_[diff])}
        assert pairs <= {(0, 2), (2, 0)}, pairs
        print(f"regrid {name}: {int(diff.sum())} of {diff.size} cells swap outcome 0 <-> 2 at the floor")
    dt = on.cfl_dt()
    on.step(dt)
    sn.step(dt)
    err = energy_scaled(sn.cons(), on.cons(), on.grid)
    print(f"regrid {name} ({form}), {g.nb} -> {len(new)} leaves: energy-scaled error after a step {err.tolist()}")
    assert np.all(err <= tol), ("step", err)


def _ct_case(name):
    from problems import ct
    from tests.test_oracle_ct_amr import _amr_field, _box
    from tests.test_oracle_ct_regrid import _coarsen_root, _refine_root, _root
    if name == "amr_torus":
        g = pb.amr_torus(root=(4, 2, 2), nblock=8).with_(divb="ct")
        P = pb.fm_torus_prims(g)
        return g, P, ct.fm_torus_faces(g, P), None
    ndim = 2 if name == "box2d" else 3
    g = _box(ndim)
    # refine the coarse root block beside the refined one and coarsen that one
    new = _coarsen_root(g.with_(blocks=_refine_root(g, _root(ndim, 1))), _root(ndim, 0))
    return g, pb.random_periodic_prims(g, jump=False), _amr_field(g, amp=0.15), new


@pytest.mark.parametrize("name,form,tol", [("box2d", "fp64", 1e-12), ("box3d", "fp64", 1e-12),
                                           ("amr_torus", "fp64", 1e-12), ("box3d", "mixed", 1e-5),
                                           ("amr_torus", "mixed", 1e-5)])
def test_regrid_with_constrained_transport_matches_oracle(gb, name, form, tol):
    """Constrained transport: the transferred face fields within 1e-12 of the
    largest face (both forms: the face transfer is FP64 arithmetic), the
    conserved state as in the cleaning form, every cell's divergence and the
    level boundaries at round-off, and one step on the new grid."""
    from problems import ct
    from tests.test_gpu_ct import _dxmin
    from tests.test_gpu_parity import energy_scaled
    g, P, F, new = _ct_case(name)
    s = gb.Solver(g, form)
    s.set_prims(P)
    s.set_faces(F)
    o = oracle.Oracle(g)
    o.set_prims(P)
    o.set_faces(F)
    if new is None:
        new = o.regrid_plan(o.estimate(), 0.3, 0.05, 2)
    assert not np.array_equal(new, np.asarray(g.blocks))
    on = o.regridded(new)
    sn = s.regridded(new)
    fg, fo = sn.faces(), on.faces()
    scale = np.abs(fo).max()
    assert np.abs(fg - fo).max() <= 1e-12 * scale, np.abs(fg - fo).max() / scale
    assert np.abs(ct.face_divergence(on.grid, fg)).max() <= 1e-12 * scale / _dxmin(on.grid)
    assert ct.level_face_mismatch(on.grid, fg) <= 1e-13 * scale
    err = energy_scaled(sn.cons(), on.cons(), on.grid)
    assert np.all(err <= tol), ("transfer", err)
    dt = on.cfl_dt()
    on.step(dt)
    sn.step(dt)
    err = energy_scaled(sn.cons(), on.cons(), on.grid)
    assert np.all(err <= tol), ("step", err)
    fg = sn.faces()
    assert np.abs(ct.face_divergence(on.grid, fg)).max() <= 1e-12 * scale / _dxmin(on.grid)
    print(f"CT regrid {name} ({form}), {g.nb} -> {len(new)} leaves: energy-scaled error after a step {err.tolist()}")


def test_regrid_with_constrained_transport_arguments(gb):
    """Forms must agree (constrained transport into cleaning is refused), and the
    faces must be loaded first."""
    from tests.test_oracle_ct_amr import _amr_field, _box
    from tests.test_oracle_ct_regrid import _refine_root, _root
    g = _box(2)
    P = pb.random_periodic_prims(g, jump=False)
    s = gb.Solver(g)
    s.set_prims(P)
    new = _refine_root(g, _root(2, 1))
    with pytest.raises(gb.BhacError) as e:
        s.regridded(new)
    assert e.value.status == 4
    s.set_faces(_amr_field(g))
    glm = gb.Solver(g.with_(divb="glm", blocks=new))
    with pytest.raises(gb.BhacError) as e:
        gb.bhac_regrid_transfer(s.ctx, glm.ctx)
    assert e.value.status == 1
