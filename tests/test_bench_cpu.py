"""Host logic of bench.py on CPU: the traffic figure attached to the
roofline, and the growth of the CPU-baseline sample toward its time target."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


class _Fake:
    """A workload whose oracle sample costs a fixed 0.5 s plus 1 µs per row."""

    def __init__(self, rows=10**9):
        self._rows = rows
        self.calls = []

    def rows(self):
        return self._rows

    def oracle_sample(self, rows):
        self.calls.append(rows)
        return 0.5 + rows * 1e-6, f"{rows} rows"

    def traffic(self):
        return ("k", 123, "profiles/x.md")


def test_traffic_only_for_the_captured_kernel():
    W = _Fake()
    assert bench.traffic_of(W, "k") == {"traffic": 123, "traffic_source": "profiles/x.md"}
    assert bench.traffic_of(W, "other") == {"traffic": None}
    assert bench.traffic_of(object(), "k") == {"traffic": None}


def test_cpu_baseline_sample_grows_past_a_fixed_cost(monkeypatch):
    import oracle
    monkeypatch.setattr(oracle, "build", lambda *a, **k: None)
    W = _Fake()
    r = bench.cpu_baseline(W, target_s=12.0)
    # a 1M-row sample looks slow (1.5 s) because of the fixed cost; the
    # sample grows until it takes at least half the target
    assert W.calls[0] == 1_000_000 and W.calls[-1] > W.calls[0]
    assert r["seconds"] >= 6.0 and r["cores"] == 1 and r["kind"] == "oracle"
    assert abs(r["value"] - W.calls[-1] / r["seconds"]) < 1e-6 * r["value"]


def test_cpu_baseline_stops_at_the_whole_workload(monkeypatch):
    import oracle
    monkeypatch.setattr(oracle, "build", lambda *a, **k: None)
    W = _Fake(rows=3_000_000)
    bench.cpu_baseline(W, target_s=60.0)
    assert max(W.calls) == 3_000_000
