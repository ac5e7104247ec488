"""Autotuner host logic: graph classes, candidate grid, the JSON table."""
import json

from paper_2404_00270_gb300 import autotune as A


def test_graph_class_buckets():
    assert A.graph_class(1 << 20, 31_400_000, 39_614) == A.graph_class(1 << 20, 31_000_000, 40_000)
    assert A.graph_class(1 << 20, 31_400_000, 39_614) != A.graph_class(4098, 16_384, 64)
    assert A.graph_class(4098, 16_384, 64).startswith("n12-d2-")


def test_candidates_cover_every_knob():
    c = list(A.candidates(152))
    assert len(c) == 162
    for key in A.KNOBS:
        assert len({x[key] for x in c}) > 1


def test_table_roundtrip(tmp_path, monkeypatch):
    path = tmp_path / "t.json"
    t = A.Table(str(path))
    t.record("n20-d5-h10", {"gr_ratio": 2.0, "small_tile": 4}, 9.0)
    t.record("n20-d5-h10", {"gr_ratio": 0.5, "small_tile": 16}, 12.0)   # slower: ignored
    t.save()
    data = json.loads(path.read_text())
    assert data["n20-d5-h10"]["options"] == {"gr_ratio": 2.0, "small_tile": 4}
    assert A.Table(str(path)).entries == data
