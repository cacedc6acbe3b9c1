"""Host-side logic of the batched disorder sweep (no device needed): the 64-point workload and
its grouping into one handle per (D, chi)."""
from inputs import DISORDER_SWEEP, disorder_sweep_points
from paper_1910_11359_gb300.sweep import group_points


def test_disorder_sweep_points():
    pts = disorder_sweep_points(DISORDER_SWEEP["n"])
    assert len(pts) == 64
    assert abs(pts[0]["h"] - 0.5) < 1e-15 and abs(pts[-1]["h"] - 16.0) < 1e-15
    assert {p["D"] for p in pts} <= {2, 3, 4} and {p["V"] for p in pts} <= {0.0, 1.0}
    assert all(p["chi"] == 2 * p["D"] ** 2 for p in pts)
    assert pts == disorder_sweep_points(DISORDER_SWEEP["n"])          # seeded


def test_group_points_partitions_by_shape():
    pts = disorder_sweep_points(64)
    groups = group_points(pts)
    seen = sorted(i for idx in groups.values() for i in idx)
    assert seen == list(range(64))
    for (D, chi), idx in groups.items():
        assert all(pts[i]["D"] == D and pts[i]["chi"] == chi for i in idx)
        assert idx == sorted(idx)                                      # input order kept
