"""Host logic of the serving loop that needs no GPU."""
from paper_2404_00270_gb300.serve import admission, footprint_estimate, latency_summary, max_overlap


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


def test_max_overlap_of_device_intervals():
    class _D:
        def __init__(self, a, b):
            self.device_ns = (a, b)
    assert max_overlap([_D(0, 10), _D(10, 20), _D(20, 30)]) == 1   # touching ends do not overlap
    assert max_overlap([_D(0, 10), _D(5, 15), _D(6, 7), _D(14, 30)]) == 3
    assert max_overlap([]) == 0


def test_admission_rejects_what_can_never_fit():
    assert admission(101, 0, 100, busy=False) == "reject"
    assert admission(101, 0, 100, busy=True) == "reject"
    assert admission(100, 0, 100, busy=False) == "admit"
    assert admission(60, 50, 100, busy=True) == "wait"
    assert admission(50, 50, 100, busy=True) == "admit"
    assert admission(60, 50, 100, busy=False) == "admit"   # nothing in flight: its bytes are free again


def test_latency_summary_skips_rejected():
    class _X:
        def __init__(self, a, d, rej=None):
            self.arrival, self.done, self.rejected = a, d, rej
    s = latency_summary([_X(0.0, 0.01), _X(0.0, 0.5, "too big")])
    assert s["solves"] == 1 and abs(s["max_ms"] - 10.0) < 1e-9
