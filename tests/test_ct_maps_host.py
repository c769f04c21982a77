"""The library's host-built constrained-transport ring maps (the ones
bhac_init_grid uploads) against the oracle's ring faces, on the CPU: the
library applies its maps to the owned faces on the host
(bhac_ct_ring_faces_host) and the result must equal the oracle's ring faces
bit for bit, on uniform and two-level boxes in 2-D and 3-D (periodic and
outflow) and on the three-level torus (polar axis, phi + pi).  No device
work; the library is loaded but runs no kernel."""
import numpy as np
import pytest

import oracle
import problems as pb
from problems import ct
from tests.test_oracle_ct_amr import _amr_field, _box


def _grids():
    yield "box2d", pb.periodic_box(ndim=2, nblock=8, nroot=2).with_(divb="ct")
    yield "torus3d", pb.torus_3d(nroot=(4, 3, 2), nblock=(8, 8, 8)).with_(divb="ct")
    yield "torus2d", pb.torus_2d(nblock=8, nroot=(4, 4)).with_(divb="ct")
    yield "amr_box2d", _box(2)
    yield "amr_box2d_outflow", _box(2, bc="outflow")
    yield "amr_box3d", _box(3)
    yield "amr_torus", pb.amr_torus(root=(4, 2, 2), nblock=8).with_(divb="ct")


@pytest.mark.parametrize("name", [n for n, _ in _grids()])
def test_library_ring_maps_equal_the_oracle_ring_faces(name):
    import paper_2108_12240_gb300 as gb
    g = dict(_grids())[name]
    if g.coords == "cart":
        P = pb.random_periodic_prims(g, jump=False)
        F = _amr_field(g) if g.nlevels > 1 else ct.random_potential_faces(g)
    else:
        P = pb.fm_torus_prims(g)
        F = ct.fm_torus_faces(g, P)
    o = oracle.Oracle(g)
    o.set_prims(P)
    o.set_faces(F)
    got = gb.bhac_ct_ring_faces_host(g, o.faces())
    for d in range(g.ndim):
        ref = o.ring_faces(d)
        assert np.array_equal(got[d], ref), (name, d, np.abs(got[d] - ref).max())


def test_library_ring_maps_reject_a_level_jump():
    import paper_2108_12240_gb300 as gb
    blocks = [(0, 1, 0, 0), (0, 0, 1, 0), (0, 1, 1, 0), (1, 0, 0, 0), (1, 1, 0, 0), (1, 0, 1, 0),
              (2, 2, 2, 0), (2, 3, 2, 0), (2, 2, 3, 0), (2, 3, 3, 0)]
    g = pb.periodic_box(ndim=2, nblock=8, nroot=2).with_(nlevels=3, blocks=np.asarray(blocks, dtype=np.int32),
                                                         divb="ct")
    with pytest.raises(gb.BhacError) as e:
        gb.bhac_ct_ring_faces_host(g, np.zeros(ct.face_count(g)))
    assert e.value.status == 1
