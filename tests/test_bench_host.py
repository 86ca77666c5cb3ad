"""Host-side arithmetic of bench.py on CPU: the leaf-vertex count of a node
tree, the algorithmic bytes per launch, the critical-path split of a stage
profile and the DRAM-traffic lookup with its source-hash check. Every
expected value is worked out by hand from the definitions in the comments."""
import hashlib
import json
import os

import pytest

import bench


@pytest.mark.parametrize("sizes, expected", [
    ([5], 5),                                  # one node: the root is a leaf
    ([2, 3, 0, 1, 1, 0, 0], 2),                # leaves 3 and 4 (1 vertex each); node 1 has vertices below
    ([0, 4, 0], 4),                            # an empty root, one non-empty child
    ([1, 0, 0, 2, 0, 0, 0], 2),                # node 3 under an empty node 1: only it is a leaf
    ([0, 0, 0], 0),
])
def test_leaf_vertex_count(sizes, expected):
    assert bench.leaf_vertex_count(sizes) == expected


def test_stage_bytes_per_launch():
    n, k, leaf = 1000, 10, 600
    stage_n = {"nd_bisect": 4, "md_small": 2, "md_mid": 1, "patch_bfs": 3, "symbolic": 5, "graph": 1}
    # per patch and per launch: 120 B a patch
    assert bench.stage_bytes_per_launch("nd_bisect", n, k, stage_n, leaf) == 120 * k
    # per step, split over the stage's launches: leaves' vertices at 32 B
    assert bench.stage_bytes_per_launch("md_small", n, k, stage_n, leaf) == 32 * leaf / 2
    # separators: the vertices outside the leaves
    assert bench.stage_bytes_per_launch("md_mid", n, k, stage_n, leaf) == 32 * (n - leaf) / 1
    # a Voronoi search moves 60 B a vertex in every launch
    assert bench.stage_bytes_per_launch("patch_bfs", n, k, stage_n, leaf) == 60 * n
    assert bench.stage_bytes_per_launch("symbolic", n, k, stage_n, leaf) == 60 * n / 5
    # no launches, or no byte model: no figure
    assert bench.stage_bytes_per_launch("quotient", n, k, stage_n, leaf) is None
    assert bench.stage_bytes_per_launch("patch_other", n, k, {"patch_other": 2}, leaf) is None


def test_critical_path():
    ms = {"graph": 0.2, "symbolic": 1.0, "md_small": 0.8, "md_mid": 3.0, "md_large": 0.5, "join_wait": 0.1}
    cp = bench.critical_path(ms)
    assert cp["handle_stream"] == pytest.approx(0.2 + 1.0 + 0.8)      # aux stages and the wait excluded
    assert cp["join_wait"] == pytest.approx(0.1)
    assert cp["auxiliary_streams"] == pytest.approx(3.5)
    assert cp["dominant"] == "symbolic" and cp["dominant_contribution"] == pytest.approx(1.0)
    # a wait longer than every stage of the handle's stream makes the longer
    # auxiliary stage the dominant one, counted by the wait alone
    ms["join_wait"] = 2.0
    cp = bench.critical_path(ms)
    assert cp["dominant"] == "md_mid" and cp["dominant_contribution"] == pytest.approx(2.0)


def test_measured_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    entry = {"stage": "symbolic", "workload": "w", "dram_bytes_per_launch": 1234, "source": "k.cu",
             "source_sha1": hashlib.sha1(src.read_bytes()).hexdigest()}
    (tmp_path / "profiles" / "kernel_traffic.json").write_text(json.dumps({"entries": [entry]}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("symbolic", "w") == 1234.0
    assert bench.measured_traffic("symbolic", "other") is None      # no record for this workload
    assert bench.measured_traffic("nd_bisect", "w") is None
    src.write_text("__global__ void k() { /* changed */ }\n")       # kernel changed since the capture
    assert bench.measured_traffic("symbolic", "w") is None


def test_committed_traffic_records_are_well_formed():
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "kernel_traffic.json")))
    for e in d["entries"]:
        assert e["stage"] in bench.STAGES
        assert e["dram_bytes_per_launch"] > 0
        assert os.path.exists(os.path.join(bench.ROOT, e["source"]))
        assert len(e["source_sha1"]) == 40 and "--clock-control none" in e["command"]
