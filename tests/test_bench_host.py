"""Host-side pieces of bench.py that need no GPU: the serving latency
statistics and the workload description."""
import numpy as np

import bench


def test_latency_stats():
    arrival = {0: 0.0, 1: 0.5, 2: 1.0, 3: 1.2}
    done = {0: 0.010, 1: 0.530, 2: 1.002, 3: 1.300}
    st = bench.latency_stats(arrival, done)
    lat = np.array([10.0, 30.0, 2.0, 100.0])
    assert st["count"] == 4
    assert abs(st["p50_ms"] - np.percentile(lat, 50)) < 1e-9
    assert abs(st["p99_ms"] - np.percentile(lat, 99)) < 1e-9
    assert abs(st["max_ms"] - 100.0) < 1e-9
    assert abs(st["solves_per_s"] - 4 / 1.3) < 1e-9
    # worst latency per arrival second: arrivals 0.0, 0.5 in second 0; 1.0, 1.2 in 1
    assert st["max_ms_by_arrival_second"] == [30.0, 100.0]
    assert bench.latency_stats({}, {}) == {"count": 0}


def test_workload_config_names_the_workload():
    cfg = bench.workload_config()
    assert "TRSM" in cfg["workload"] and "TRMM" in cfg["workload"]
    assert cfg["l2"].startswith("inputs larger than L2")
