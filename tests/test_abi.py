"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point the public header declares, sizes arenas and rejects
invalid descriptions."""
import os
import re

import numpy as np
import pytest

import paper_2108_12240_gb300 as gb
import problems as pb

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "bhac_gb300.h")


def declared_functions():
    text = open(HDR).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bhac_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_entry_point():
    names = declared_functions()
    assert "bhac_step" in names and "bhac_init_grid" in names and len(names) >= 12
    L = gb.lib()
    for n in names:
        assert hasattr(L, n), n


def test_python_binding_has_every_declared_entry_point():
    """The binding mirrors the header name for name (marshalling only)."""
    missing = [n for n in declared_functions() if not callable(getattr(gb, n, None))]
    assert not missing, missing
    assert set(declared_functions()) <= set(gb.__all__)


def test_query_sizes_counts_state_and_tables():
    g = pb.torus_3d(nroot=(2, 2, 2))
    n64 = gb.bhac_query_sizes(gb.desc_of(g, "fp64"), gb.blocks_of(g))
    n32 = gb.bhac_query_sizes(gb.desc_of(g, "mixed"), gb.blocks_of(g))
    cells_g = 22 ** 3 * g.nb
    cells_i = 16 ** 3 * g.nb
    # two ghosted FP64 primitive buffers, two conserved buffers and the two
    # staging arrays of host transfers at least
    assert n64 >= 8 * 9 * (2 * cells_g + 4 * cells_i)
    assert n32 >= n64 + 4 * 9 * 2 * cells_g


@pytest.mark.parametrize("bad", [
    dict(ndim=4), dict(nx=(2, 16, 1)), dict(nroot=(0, 1, 1)), dict(gamma_ad=1.0), dict(cfl=0.0),
    dict(bc=(("axis", "axis"), ("periodic", "periodic"), ("periodic", "periodic"))),
])
def test_invalid_descriptions_are_rejected(bad):
    g = pb.shock_tube_2d(nblock=16, nroot=2)
    g = g.with_(**bad)
    with pytest.raises(gb.BhacError) as e:
        gb.bhac_query_sizes(gb.desc_of(g), gb.blocks_of(pb.shock_tube_2d(nblock=16, nroot=2)))
    assert e.value.status == 1


def test_status_strings():
    assert gb.status_string(0) == "ok"
    assert gb.status_string(3) == "arena too small or device allocation failed"


def test_empty_and_inconsistent_block_lists_are_rejected():
    """No blocks, a block outside the root grid, a duplicate block, and a
    level beyond the grid's levels: BHAC_ERR_ARG before any device work."""
    g = pb.shock_tube_2d(nblock=16, nroot=2)
    d = gb.desc_of(g)
    for blocks in ([], [(0, 0, 0, 0), (0, 2, 0, 0)], [(0, 0, 0, 0), (0, 0, 0, 0)], [(3, 0, 0, 0)]):
        arr = (gb.BlockDesc * len(blocks))()
        for n, (lev, ix, iy, iz) in enumerate(blocks):
            arr[n].level, arr[n].ix, arr[n].iy, arr[n].iz = lev, ix, iy, iz
        with pytest.raises(gb.BhacError) as e:
            gb.bhac_query_sizes(d, arr)
        assert e.value.status == 1, blocks



def test_constrained_transport_descriptors():
    """Constrained transport adds the face fields, the ring-extended fluxes and
    the ring map to the arena, in either form; with refinement levels also the
    edge EMFs and the correction maps.  Its level maps need neighbouring
    leaves (across faces, edges and corners) to differ by at most one level:
    a grid that breaks that is rejected before any device work, although the
    cleaning form accepts it."""
    g = pb.periodic_box(ndim=3, nblock=8, nroot=2)
    n_glm = gb.bhac_query_sizes(gb.desc_of(g), gb.blocks_of(g))
    n_ct = gb.bhac_query_sizes(gb.desc_of(g.with_(divb="ct")), gb.blocks_of(g))
    faces = g.nb * 3 * 9 * 10 * 10  # ring-extended faces per direction per block
    assert n_ct >= n_glm + 8 * faces * (2 + 9)
    n_ct_mixed = gb.bhac_query_sizes(gb.desc_of(g.with_(divb="ct"), "mixed"), gb.blocks_of(g))
    assert n_ct_mixed >= gb.bhac_query_sizes(gb.desc_of(g, "mixed"), gb.blocks_of(g)) + 8 * faces * (2 + 9)
    amr = pb.amr_torus(root=(4, 2, 2), nblock=8)
    n_amr = gb.bhac_query_sizes(gb.desc_of(amr), gb.blocks_of(amr))
    edges = amr.nb * 3 * 8 * 9 * 9
    assert gb.bhac_query_sizes(gb.desc_of(amr.with_(divb="ct")), gb.blocks_of(amr)) >= n_amr + 8 * (
        amr.nb * 3 * 9 * 10 * 10 * (2 + 9) + edges)
    blocks = [(0, 1, 0, 0), (0, 0, 1, 0), (0, 1, 1, 0), (1, 0, 0, 0), (1, 1, 0, 0), (1, 0, 1, 0),
              (2, 2, 2, 0), (2, 3, 2, 0), (2, 2, 3, 0), (2, 3, 3, 0)]  # level 2 next to level 0
    jump = pb.periodic_box(ndim=2, nblock=8, nroot=2).with_(nlevels=3, blocks=np.asarray(blocks, dtype=np.int32))
    assert gb.bhac_query_sizes(gb.desc_of(jump), gb.blocks_of(jump)) > 0
    with pytest.raises(gb.BhacError) as e:
        gb.bhac_query_sizes(gb.desc_of(jump.with_(divb="ct")), gb.blocks_of(jump))
    assert e.value.status == 1


def test_imex_flag_is_validated():
    g = pb.shock_tube_2d(nblock=16, nroot=2)
    d = gb.desc_of(g)
    d.imex = 2
    with pytest.raises(gb.BhacError) as e:
        gb.bhac_query_sizes(d, gb.blocks_of(g))
    assert e.value.status == 1


def test_c2p_solver_is_validated():
    """The primary inversion is BHAC_C2P_NEWTON (0) or BHAC_C2P_NK (1); the
    Newton-Krylov choice sizes the same arena, another value is rejected."""
    g = pb.shock_tube_2d(nblock=16, nroot=2)
    n0 = gb.bhac_query_sizes(gb.desc_of(g), gb.blocks_of(g))
    assert gb.bhac_query_sizes(gb.desc_of(g.with_(c2p="nk")), gb.blocks_of(g)) == n0
    for bad in (-1, 2):
        d = gb.desc_of(g)
        d.c2p_solver = bad
        with pytest.raises(gb.BhacError) as e:
            gb.bhac_query_sizes(d, gb.blocks_of(g))
        assert e.value.status == 1
