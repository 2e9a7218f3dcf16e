"""Host-side helpers of bench.py that need no GPU: the serving record's
latency by request size."""
import bench


def test_latency_by_size_bands_and_percentiles():
    edges = [500, 2_000, 99_999, 100_000, 150_000, 999_999, 1_000_000, 5_000_000]
    lat = [1.0, 3.0, 2.0, 10.0, 12.0, 11.0, 90.0, 70.0]
    out = bench.latency_by_size(edges, lat)
    assert list(out) == ["<100k edges", "100k-1M edges", ">=1M edges"]
    assert out["<100k edges"] == {"requests": 3, "p50_ms": 2.0, "p99_ms": 3.0}
    assert out["100k-1M edges"] == {"requests": 3, "p50_ms": 11.0, "p99_ms": 12.0}
    assert out[">=1M edges"]["requests"] == 2 and out[">=1M edges"]["p99_ms"] == 90.0
    assert sum(b["requests"] for b in out.values()) == len(edges)


def test_latency_by_size_leaves_out_empty_bands():
    assert bench.latency_by_size([], []) == {}
    assert list(bench.latency_by_size([10, 20], [1.0, 2.0])) == ["<100k edges"]
