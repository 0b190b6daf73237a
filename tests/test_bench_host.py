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


def test_auto_path_description_follows_the_plan():
    # the bench's description of the automatic TRSM path agrees with the
    # library's plan (thin leaves and their size, as the plan dump shows)
    from paper_2504_13821_gb300 import debug_plan
    for k, n in ((16384, 16384), (16384, 1024), (16384, 256), (16384, 128), (8192, 512),
                 (4096, 128), (4096, 256), (2048, 256), (16384, 2048)):
        desc = bench.auto_path_desc(k, n)
        sizes = {s["b"] for s in debug_plan("S", "L", "L", "N", "N", k, n, 4, 0, 0)
                 if s["kind"] == "thin"}
        if sizes:
            assert desc.startswith(f"TRSM leaves of {sizes.pop()} rows as thin solves"), (k, n)
        else:
            assert not desc.startswith("TRSM leaves of"), (k, n)


def test_triangle_upload_bytes():
    # one rectangle of rows j0..k-1 per 256-column block
    assert bench.triangle_upload_bytes(256, 4) == 256 * 256 * 4
    assert bench.triangle_upload_bytes(300, 8) == (300 * 256 + 44 * 44) * 8
    k = 16384
    tri = k * (k + 1) // 2
    assert tri * 4 < bench.triangle_upload_bytes(k, 4) < (tri + 128 * k) * 4
