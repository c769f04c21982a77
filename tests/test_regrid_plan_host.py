"""The library's regrid plan (host code behind the C ABI) against the
oracle's on the same leaf lists and block errors: identical leaf lists, over
random multi-level cases on periodic boxes and through the polar axis.  The
oracle's plan is pinned in test_oracle_regrid.  CPU only (no device work)."""
import numpy as np
import pytest

import oracle
import paper_2108_12240_gb300 as gb
import problems as pb


def _box(ndim):
    return pb.periodic_box(ndim=ndim, nblock=4, nroot=3 if ndim == 3 else 4).with_(nlevels=5)


@pytest.mark.parametrize("case,seed", [("box2", 1), ("box2", 39), ("box3", 3), ("torus", 9)])
def test_library_plan_equals_oracle_plan(case, seed):
    rng = np.random.default_rng(seed)
    if case == "torus":
        g = pb.amr_torus(root=(4, 2, 2), nblock=4)
        maxl = 2
    else:
        g = _box(2 if case == "box2" else 3)
        maxl = 4
    blocks = np.asarray(g.blocks)
    for _ in range(5):
        gg = g.with_(blocks=blocks)
        err = rng.random(len(blocks)) ** 3
        ref = oracle.Oracle(gg).regrid_plan(err, 0.5, 0.2, maxl)
        got = gb.bhac_regrid_plan(gb.desc_of(gg), gb.blocks_of(gg), err, 0.5, 0.2, maxl)
        assert np.array_equal(got, ref)
        blocks = got
        if len(blocks) > 3000:
            break


def test_plan_rejects_bad_input():
    g = _box(2)
    err = np.zeros(g.nb)
    with pytest.raises(gb.BhacError):
        gb.bhac_regrid_plan(gb.desc_of(g), gb.blocks_of(g), err, 0.5, 0.2, 9)  # beyond nlevels
    dup = g.with_(blocks=np.concatenate([g.blocks, g.blocks[:1]]))
    with pytest.raises(gb.BhacError):
        gb.bhac_regrid_plan(gb.desc_of(dup), gb.blocks_of(dup), np.zeros(dup.nb), 0.5, 0.2, 2)
