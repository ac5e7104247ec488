"""Host logic of the serving loop that needs no GPU."""
from paper_2404_00270_gb300.serve import footprint_estimate, latency_summary


class _R:
    def __init__(self, a, d):
        self.arrival, self.done = a, d


def test_latency_summary_percentiles():
    reqs = [_R(i * 0.01, i * 0.01 + 0.001 * (i + 1)) for i in range(100)]
    s = latency_summary(reqs)
    assert s["solves"] == 100
    assert abs(s["p50_ms"] - 51.0) < 1.01 and abs(s["p99_ms"] - 100.0) < 1.01
    assert abs(s["max_ms"] - 100.0) < 1e-9
    assert abs(s["makespan_s"] - (0.99 + 0.1)) < 1e-9
    assert latency_summary([]) == {}


def test_footprint_grows_with_size():
    assert footprint_estimate(10, 10) < footprint_estimate(10, 20) < footprint_estimate(20, 20)
