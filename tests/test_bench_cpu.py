"""Host-side pieces of bench.py: the oracle baseline of the batch workload
(a sequential pass and a spawned worker pool over the same instances)."""
import bench


def test_batch_cpu_baseline_small_mix():
    specs = [("grid", 32, 1000), ("bip", 1024, 4, 1001), ("grid", 40, 1002), ("bip", 2048, 8, 1003)]
    r = bench.batch_cpu_baseline(specs, 4)
    assert r["kind"] == "oracle" and r["cores"] == 1 and r["unit"] == "solves/s"
    assert r["value"] > 0 and r["all_cores"]["value"] > 0 and r["all_cores"]["cores"] >= 1
    assert "4 evenly spaced instances" in r["sample"]
