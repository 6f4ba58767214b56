"""Host-side arithmetic of bench.py that feeds its JSON line (CPU only): the
logical product count of a solve, the whole-job throughput, the roofline's
DRAM traffic per launch from an ncu capture (only when it was taken on the
current kernel source and at the same size), and the peak table."""
import hashlib
import json

import pytest

import bench


def test_logical_products_of_a_solve():
    # forward M squares, M - ceil(M/k) recomputed squares, M adjoint products Y X
    n = 16384
    assert bench.logical_flops(n, 54, 4) == 148 * 2.0 * n ** 3
    assert bench.logical_flops(n, 54, 1) == 108 * 2.0 * n ** 3    # history kept: no recompute
    assert bench.logical_flops(n, 53, 4) == (53 + 39 + 53) * 2.0 * n ** 3
    assert bench.logical_flops(128, 1, 4) == 2 * 2.0 * 128 ** 3    # one step: nothing to recompute


def test_whole_job_value_uses_the_slowest_rank():
    # two ranks, each 1e15 flop, the slower one took 1000 ms: 2 PFLOP/s in TFLOP/s
    assert bench.whole_job_tflops(2, 1e15, 1000.0) == pytest.approx(2000.0)
    assert bench.whole_job_tflops(1, 1e15, 500.0) == pytest.approx(2000.0)


def _capture(path, sha, n=16384, sq=(8.0, 2.0), pl=(20.0, 1.0)):
    d = {"kernel_sha256": sha, "n": n,
         "square": {"read_bytes": sq[0], "write_bytes": sq[1]},
         "plain": {"read_bytes": pl[0], "write_bytes": pl[1]}}
    path.write_text(json.dumps(d))


def test_traffic_is_the_launch_mix_average(tmp_path, monkeypatch):
    sha = hashlib.sha256(open(bench.TC_SOURCE, "rb").read()).hexdigest()
    f = tmp_path / "traffic.json"
    _capture(f, sha)
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    # M = 54, k = 4: 94 squares (10 bytes each) and 54 plain products (21 bytes each)
    assert bench.traffic_per_launch(16384, 54, 4) == pytest.approx((94 * 10.0 + 54 * 21.0) / 148)
    # another size, another kernel source or no capture: no traffic figure
    assert bench.traffic_per_launch(8192, 54, 4) is None
    _capture(f, "0" * 64)
    assert bench.traffic_per_launch(16384, 54, 4) is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.json"))
    assert bench.traffic_per_launch(16384, 54, 4) is None


def test_peak_table_has_the_roofline_denominators():
    p, kind = bench.peaks()
    assert kind in ("measured", "fallback")
    for key in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained"):
        assert p[key] > 0
