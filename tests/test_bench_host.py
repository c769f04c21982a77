"""Host-side logic of the benchmark line (no GPU): the source fingerprint that
ties a recorded DRAM-traffic figure to the code it was measured on, and the
lookup that reports the figure only for the matching sources, workload, form
and launch shape."""
import pytest

import bench


def test_code_only_ignores_comments_and_layout():
    a = "int f(int x) {  // one\n  return x + 1; /* two\n lines */ }\n"
    b = "int f(int x) {\n\n    return x + 1;   }"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(a.replace("x + 1", "x + 2"))


def test_fingerprint_is_stable_and_hex():
    f = bench.kernel_fingerprint()
    assert f == bench.kernel_fingerprint()
    assert len(f) == 64 and int(f, 16) >= 0


def test_shape_key_leaves_out_the_persistent_schedule():
    """The persistent schedule does not change a launch's bytes; the z parts
    do (each part recomputes the z faces at its bottom)."""
    ls = {"tx": 16, "ty": 16, "threads": 256, "persistent": 2, "min_ctas": 2, "producer_warps": 0, "z_parts": 1}
    assert bench.shape_key(ls) == "16x16/256/minctas2/producers0/zparts1"
    assert bench.shape_key(dict(ls, persistent=0)) == bench.shape_key(ls)
    assert bench.shape_key(dict(ls, z_parts=2)) != bench.shape_key(ls)


@pytest.fixture
def record(tmp_path, monkeypatch):
    def write(sha, workload="torus_3d_large"):
        p = tmp_path / "traffic.txt"
        p.write_text("# header: with a colon\n"
                     f"sources_sha256: {sha}\n"
                     f"workload: {workload}\n"
                     "traffic mixed 16x16/256/minctas2/producers0/zparts1: 15887270768  (a) stage1 ...\n"
                     "traffic fp64 16x16/256/minctas1/producers0/zparts1: 13958643712  (a) stage1 ...\n")
        monkeypatch.setattr(bench, "TRAFFIC_FILE", str(p))
    return write


def test_recorded_traffic_matches_sources_workload_form_and_shape(record):
    record(bench.kernel_fingerprint())
    assert bench.recorded_traffic("torus_3d_large", "mixed", "16x16/256/minctas2/producers0/zparts1") == 15887270768.0
    assert bench.recorded_traffic("torus_3d_large", "fp64", "16x16/256/minctas1/producers0/zparts1") == 13958643712.0
    assert bench.recorded_traffic("torus_3d_large", "mixed", "16x16/256/minctas1/producers0/zparts1") is None
    assert bench.recorded_traffic("torus_3d", "mixed", "16x16/256/minctas2/producers0/zparts1") is None


def test_recorded_traffic_is_dropped_for_other_sources(record):
    record("0" * 64)
    assert bench.recorded_traffic("torus_3d_large", "mixed", "16x16/256/minctas2/producers0/zparts1") is None


def test_recorded_traffic_without_a_record(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.txt"))
    assert bench.recorded_traffic("torus_3d_large", "mixed", "16x16/256/minctas2/producers0/zparts1") is None


def test_fill_roofline_counts_ghost_cells_and_bytes():
    import problems as pb
    g = pb.torus_3d_large()
    r = bench.fill_roofline(g, "fp64", 1.0, 6792.1)
    assert r["ghost_cells"] == 2048 * (38 * 38 * 22 - 32 * 32 * 16)
    assert r["bytes_per_fill"] == r["ghost_cells"] * 149
    assert abs(r["achieved"] - r["bytes_per_fill"] / 1e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6792.1) < 1e-12
    m = bench.fill_roofline(pb.torus_2d(), "mixed", 0.5, None)
    assert m["ghost_cells"] == 256 * (22 * 22 - 16 * 16)
    assert m["bytes_per_fill"] == m["ghost_cells"] * 77 and m["frac"] is None
