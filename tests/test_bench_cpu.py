"""Host-side pieces of bench.py: the oracle baseline of the batch workload
(a sequential pass and a spawned worker pool over the same instances)."""
import bench


def test_batch_cpu_baseline_small_mix():
    specs = [("grid", 32, 1000), ("bip", 1024, 4, 1001), ("grid", 40, 1002), ("bip", 2048, 8, 1003)]
    r = bench.batch_cpu_baseline(specs, 4)
    assert r["kind"] == "oracle" and r["cores"] == 1 and r["unit"] == "solves/s"
    assert r["value"] > 0 and r["all_cores"]["value"] > 0 and r["all_cores"]["cores"] >= 1
    assert "4 evenly spaced instances" in r["sample"]


def test_reference_arm_prints_one_json_line():
    """`bench.py --impl reference` needs no GPU: one JSON line that carries
    the reference marker, the headline metric and unit, and a cpu_baseline
    and e2e describing the oracle run itself."""
    import json
    import os
    import subprocess
    import sys
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env,
                         timeout=600, check=True).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.metric_name("rmat26")
    assert d["unit"] == "arcs/s" and d["higher_is_better"] is True and d["steps"] == 1
    assert d["config"]["workload"] == "rmat26-maxflow-mincut" and d["config"]["scale"] == 26
    assert "R-MAT scale 18" in d["config"]["sample_per_step"]
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"] == {"value": d["value"], "unit": "arcs/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_algorithmic_bytes_per_unit():
    """Each counter of wbpr_stats is charged its own bytes per unit; a
    compaction from the candidate bitmap costs the bitmap (one bit per
    vertex) plus each candidate, a full one every vertex."""
    keys = ("arcs_scanned", "active_total", "avq_full_scans", "avq_bitmap_scans", "avq_candidates",
            "pushes", "relabels", "gr_arcs_scanned", "global_relabels")
    zero = dict.fromkeys(keys, 0)
    n = 1 << 20
    per = {"arcs_scanned": 12, "active_total": 36, "avq_full_scans": 12 * n, "avq_bitmap_scans": n // 8,
           "avq_candidates": 12, "pushes": 52, "relabels": 4, "gr_arcs_scanned": 12,
           "global_relabels": 12 * n}
    for k in keys:
        st = dict(zero, **{k: 3})
        assert bench.algorithmic_bytes(st, n) == 3 * per[k], k
    assert bench.algorithmic_bytes(zero, n, slots=1000) == 20 * 1000


def test_profiled_traffic_follows_the_solver_source(monkeypatch):
    """roofline.traffic comes from the committed ncu record only while the
    solver's device code is the one it was captured on."""
    import json
    import os
    with open(os.path.join(bench.ROOT, "profiles", "solve_kernel_rmat26.json")) as f:
        rec = json.load(f)
    prefix = rec["solver_impl_sha256_prefix"]
    monkeypatch.setattr(bench, "solver_sha", lambda: prefix + "0" * 48)
    assert bench.profiled_traffic("rmat26") == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    assert bench.profiled_traffic("rmat26") == rec["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "solver_sha", lambda: "f" * 64 if prefix[0] != "f" else "0" * 64)
    assert bench.profiled_traffic("rmat26") is None
    assert bench.profiled_traffic("no-such-workload") is None


def test_launch_count_of_the_headline_step():
    """Eleven of the library's own kernels per renumbered R-MAT step with an
    even arc count: three renumbering kernels, five builder kernels, two
    solver launches and the edge-flow kernel; two scalar tail kernels more
    for an odd half-entry count."""
    assert bench.launches_per_step(True, 1060385108) == 11
    assert bench.launches_per_step(False, 16085996) == 8
    assert bench.launches_per_step(True, 7) == 13
