"""Host-side logic of the serving loop (no GPU): footprints, request streams,
latency summaries."""
import workloads as W
from paper_1202_6130_gb300 import serve


def test_footprint_grows_with_size_and_precision():
    a = serve.footprint_bytes(64, 32, "fp32")
    b = serve.footprint_bytes(128, 64, "fp32")
    c = serve.footprint_bytes(128, 64, "fp64")
    d = serve.footprint_bytes(128, 64, "fp16s")
    assert a < b and d < b < c
    # two FP32 population buffers of a 1024x512 lattice alone are 2*9*4*N bytes
    assert serve.footprint_bytes(1024, 512, "fp32") > 2 * 9 * 4 * 1024 * 512


def test_stream_requests_are_poisson_ordered_and_bounded():
    st = W.serving_stream(rate=50.0, duration=2.0, seed=3)
    reqs = serve.requests_from_stream(st)
    assert 50 <= len(reqs) <= 150
    assert all(a.t_arrival <= b.t_arrival for a, b in zip(reqs, reqs[1:]))
    assert all(64 <= r.nx <= 2048 and 32 <= r.ny <= 1024 for r in reqs)
    assert all(1000 <= r.steps <= 20000 for r in reqs)
    assert {r.kind for r in reqs} == {"droplet", "channel"}


def test_summary_percentiles():
    rs = [serve.Result(i, "droplet", 8, 8, 10, 0.0, 0.0, float(i + 1), 0.0) for i in range(100)]
    s = serve.summarize(rs, 10.0)
    assert s["requests"] == 100 and abs(s["p50_s"] - 50.5) < 1e-9 and s["p99_s"] > 99
    assert abs(s["mlups"] - 100 * 640 / 10.0 / 1e6) < 1e-12
