"""The allocation-free CFL entry point against the arena-based one.

bhac_cfl_dt_static serves callers that cannot allocate device memory (hosts
whose device memory belongs to another allocator and that hand the library no
arena, per-step diagnostics that must not enter an allocator because
cudaMalloc can synchronise the device): it keeps its scratch in fixed
file-scope device arrays.  Here it must give the same dt as bhac_cfl_dt, within
the 1e-14 relative tolerance the CFL parity test uses, on two calls in a row,
and reject a grid with more blocks than its fixed scratch holds.  The grids
cover every metric branch of its own cell-centre metric: modified Kerr-Schild
(3-D torus, 3-level AMR torus, 2-D torus), plain Kerr-Schild coordinates
(the flat-space monopole, M = 0) and Cartesian Minkowski (the shock tube).
This file is collected last."""
import numpy as np
import pytest

import problems as pb

pytestmark = pytest.mark.gpu


def _grid(name):
    if name == "torus_3d":
        return pb.torus_3d(nroot=(4, 3, 2))
    if name == "amr_torus":
        return pb.amr_torus(root=(4, 2, 2), nblock=8)
    if name == "torus_2d":
        return pb.torus_2d(nblock=8)
    if name == "monopole_ks":
        return pb.monopole_flat_spherical(nr_blocks=4)
    return pb.shock_tube_2d()


def _prims(g):
    if g.coords == "mks":
        return pb.fm_torus_prims(g)
    if g.coords == "ks":
        return pb.monopole_prims(g)
    return pb.shock_tube_prims(g)


@pytest.mark.parametrize("grid", ["torus_3d", "amr_torus", "torus_2d", "monopole_ks", "shock_tube_2d"])
def test_static_cfl_matches_arena_cfl(grid):
    import torch

    import paper_2108_12240_gb300 as gb

    g = _grid(grid)
    P = _prims(g)
    st = torch.cuda.Stream()
    s = gb.Solver(g, stream=st)
    s.set_prims(P)
    ref = s.cfl_dt()
    prims = torch.from_numpy(np.ascontiguousarray(P)).to("cuda")
    dt = torch.zeros(2, dtype=torch.float64, device="cuda")
    # the primitives and the zeroed outputs were written on the current stream
    st.wait_stream(torch.cuda.current_stream())
    desc, blocks = gb.desc_of(g), gb.blocks_of(g)
    for call in range(2):
        gb.bhac_cfl_dt_static(desc, blocks, prims.data_ptr(), dt[call:].data_ptr(), st.cuda_stream)
    st.synchronize()
    got = dt.cpu().numpy()
    assert got[0] == pytest.approx(ref, rel=1e-14)
    assert got[1] == pytest.approx(ref, rel=1e-14)


def test_static_cfl_rejects_too_many_blocks():
    import paper_2108_12240_gb300 as gb

    g = pb.torus_3d(nblock=(4, 4, 4), nroot=(64, 16, 20))  # 20480 blocks > 16384
    with pytest.raises(gb.BhacError) as e:
        gb.bhac_cfl_dt_static(gb.desc_of(g), gb.blocks_of(g), 1, 1, 0)
    assert e.value.status == 1
