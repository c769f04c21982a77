"""Host-side rules of the Solver convenience class (no GPU): a solver lives on
the current CUDA device, because the library launches on the device current
at each call.  A device or stream of another GPU is refused before any
allocation (with one process per GPU, each rank selects its own device and
its solvers follow)."""
import pytest
import torch

import paper_2108_12240_gb300 as gb
import problems as pb


class _Stream:
    def __init__(self, idx):
        self.device = torch.device("cuda", idx)
        self.cuda_stream = 0


class _Reached(Exception):
    pass


@pytest.fixture
def on_device_3(monkeypatch):
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 3)

    def stop(*args, **kwargs):
        raise _Reached()

    # the first library call after the device checks
    monkeypatch.setattr(gb, "bhac_query_sizes", stop)


@pytest.mark.parametrize("device,stream", [(None, None), ("cuda:3", None), ("cuda", None), (None, _Stream(3))])
def test_solver_follows_the_current_device(on_device_3, device, stream):
    with pytest.raises(_Reached):
        gb.Solver(pb.torus_2d(), "fp64", device=device, stream=stream)


@pytest.mark.parametrize("device,stream", [("cuda:0", None), (None, _Stream(1))])
def test_solver_refuses_another_device(on_device_3, device, stream):
    with pytest.raises(ValueError):
        gb.Solver(pb.torus_2d(), "fp64", device=device, stream=stream)
