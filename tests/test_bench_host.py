"""Host logic of bench.py that needs no GPU: the recorded DRAM traffic of the
headline element kernel is reported only for the kernel sources it was captured
with (their SHA-256 in the record), for its own workload and in FP64."""
import importlib.util
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_host", os.path.join(HERE, "..", "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    return bench


def test_traffic_record_is_reported_for_its_kernel(monkeypatch):
    bench = load_bench()
    import re
    txt = open(bench.TRAFFIC_FILE).read()
    sha = re.search(r"sources_sha256:\s*([0-9a-f]{64})", txt).group(1)
    nbytes = int(re.search(r"traffic_bytes_per_launch:\s*(\d+)", txt).group(1))
    monkeypatch.setattr(bench, "kernel_sources_sha", lambda: sha)
    traffic, src = bench.recorded_traffic("tall192x192x384_gr1e6", "f64")
    assert traffic == nbytes > 0
    assert src.startswith("profiles/") and src.endswith(".txt")


def test_traffic_record_is_withheld_when_it_does_not_apply(monkeypatch):
    bench = load_bench()
    assert bench.recorded_traffic("tall192x192x384_gr1e6", "f32")[0] is None
    assert bench.recorded_traffic("cavity128_gr1e5", "f64")[0] is None
    monkeypatch.setattr(bench, "kernel_sources_sha", lambda: "0" * 64)
    traffic, why = bench.recorded_traffic("tall192x192x384_gr1e6", "f64")
    assert traffic is None and "changed" in why
