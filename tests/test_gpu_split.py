"""The split form of the stage (face kernel, then cell kernel on a second
stream, chunk by chunk) against the fused stage kernel and the oracle, through
the C ABI.

Both forms run the same arithmetic, so after two steps with the device time
step the conserved state, primitives and inversion statuses must agree bit for
bit, for every chunk count, persistent or per-item launch, and register bound
(min_ctas 3 applies to the face kernel only); uniform and AMR grids, 2-D and
3-D, Minkowski and modified Kerr-Schild, with and without IMEX.  One FP64 case
is also checked against the oracle at 1e-12 (energy-scaled)."""
import numpy as np
import pytest

import oracle
import problems as pb

pytestmark = pytest.mark.gpu

SHAPES = [(1, 0, 1), (3, 0, 3), (8, 2, 2), (3, 3, 3)]  # (chunks, persistent, min_ctas)


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_2108_12240_gb300 as m
    return m


def _case(name):
    if name == "torus3d":
        g = pb.torus_3d(nroot=(4, 3, 2))
        return g, pb.fm_torus_prims(g)
    if name == "amr":
        g = pb.amr_torus(root=(4, 2, 2), nblock=8)
        return g, pb.fm_torus_prims(g)
    if name == "torus2d":
        g = pb.torus_2d(nblock=16, nroot=(6, 4))
        return g, pb.fm_torus_prims(g)
    if name == "box3d_imex":
        g = pb.periodic_box(ndim=3, nblock=8, nroot=2, kappa=50.0, imex=True)
        return g, pb.random_periodic_prims(g, jump=True)
    g = pb.shock_tube_2d()
    return g, pb.shock_tube_prims(g)


def _run(gb, g, P, form, chunks, persistent, min_ctas, steps=2):
    s = gb.Solver(g, form)
    s.set_launch(8, 8, 256, persistent, min_ctas, 0)
    s.set_split(chunks)
    s.set_prims(P)
    s.cfl_dt()
    for _ in range(steps):
        s.step(0.0)
    return s.cons(), s.prims(), s.c2p_status()


@pytest.mark.parametrize("form", ["mixed", "fp64"])
@pytest.mark.parametrize("name", ["torus3d", "amr", "torus2d", "box3d_imex", "shock_tube"])
def test_split_is_the_fused_stage_bit_for_bit(gb, name, form):
    g, P = _case(name)
    ref = _run(gb, g, P, form, 0, 0, 2 if (form == "mixed" and g.ndim == 3) else 1)
    for chunks, pers, minb in SHAPES:
        got = _run(gb, g, P, form, chunks, pers, minb)
        for a, b, what in zip(got, ref, ("cons", "prims", "c2p status")):
            assert np.array_equal(a, b), (name, form, chunks, pers, minb, what)


def test_split_fp64_matches_the_oracle(gb):
    from tests.test_gpu_parity import energy_scaled
    g, P = _case("torus3d")
    s = gb.Solver(g)
    s.set_split(4)
    s.set_prims(P)
    o = oracle.Oracle(g)
    o.set_prims(P)
    for _ in range(2):
        dt = o.cfl_dt()
        assert s.cfl_dt() == pytest.approx(dt, rel=1e-13)
        o.step(dt)
        s.step(dt)
        err = energy_scaled(s.cons(), o.cons(), g)
        assert np.all(err <= 1e-12), err


def test_split_arguments_and_graph_capture(gb):
    import torch
    g, P = _case("torus2d")
    s = gb.Solver(g, stream=torch.cuda.Stream())
    for bad in (-1, 33):
        with pytest.raises(gb.BhacError) as e:
            s.set_split(bad)
        assert e.value.status == 1
    s.set_split(2)
    s.set_prims(P)
    s.cfl_dt()
    with pytest.raises(gb.BhacError) as e:
        s.capture(1)
    assert e.value.status == 4
    s.set_split(0)
    s.capture(1)  # the fused form captures again
    s.replay()
    s.stream.synchronize()
    ct = gb.Solver(pb.torus_2d(nblock=16, nroot=(6, 4)).with_(divb="ct"))
    with pytest.raises(gb.BhacError) as e:
        ct.set_split(2)
    assert e.value.status == 1


@pytest.mark.parametrize("form", ["mixed", "fp64"])
@pytest.mark.parametrize("name", ["torus3d", "amr", "box3d_imex"])
def test_z_parts_are_the_whole_columns_bit_for_bit(gb, name, form):
    """Work items cut into z parts (each recomputes the z faces at its bottom)
    give the same bits as whole columns, for a fixed part count and for the
    library's own choice; AMR grids exercise the coarse-fine face registers at
    the block's z ends."""
    g, P = _case(name)
    outs = []
    for parts in (1, 2, 4, 0):
        s = gb.Solver(g, form)
        s.set_launch(8, 8, 256, 2 if parts == 4 else 0, 0, 0)
        s.set_zsplit(parts)
        s.set_prims(P)
        s.cfl_dt()
        for _ in range(2):
            s.step(0.0)
        assert s.zsplit_in_force() == (parts if parts else s.zsplit_in_force()) >= 1
        outs.append((parts, s.cons(), s.prims()))
    for parts, c, p in outs[1:]:
        assert np.array_equal(c, outs[0][1]), (name, form, parts)
        assert np.array_equal(p, outs[0][2]), (name, form, parts)


def test_z_parts_arguments(gb):
    g, _ = _case("torus3d")
    s = gb.Solver(g)
    for bad in (-1, 3, 32):
        with pytest.raises(gb.BhacError) as e:
            s.set_zsplit(bad)
        assert e.value.status == 1
    two = gb.Solver(pb.torus_2d(nblock=16, nroot=(6, 4)))
    with pytest.raises(gb.BhacError) as e:
        two.set_zsplit(2)
    assert e.value.status == 1
