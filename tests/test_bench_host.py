"""Host arithmetic of bench.py (CPU): the roofline fields follow from the
algorithmic byte model and the event timing, the recorded ncu traffic table
matches the byte model at the instances that were captured, and the extra
attempt rates take the median timed step."""
import json
import os
import sys

import pytest

from tests.conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_roofline_fields_follow_from_bytes_and_time():
    m, n, nnz = 2_000_000, 5_000_000, 29_947_234
    kt_ms = [248.0e-3 * 60, 164.0e-3 * 60]  # summed event times (ms) of 60 sampled launches each
    kt_n = [60, 60]
    r = bench.roofline("powerlaw", m, n, nnz, kt_ms, kt_n, {"sm_mhz": 2070.0}, "double")
    pb, db = bench.kernel_bytes(m, n, nnz, 8)
    peak, _ = bench.measured_peaks()
    assert r["kernel"].startswith("primal_step_kernel<double>")
    assert r["algorithmic_bytes_per_launch"] == pb and r["other_kernel_bytes_per_launch"] == db
    assert r["achieved"] == pytest.approx(pb / 248.0e-6 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / peak) and r["peak"] == peak
    t = bench.NCU_TRAFFIC[("powerlaw", "primal", "double")]
    assert r["traffic"] == pytest.approx(t[0] * pb / t[1])
    fp = r["fp64_alu"]
    assert fp["peak"] == pytest.approx(152 * 2 * 2070e6 / 1e9)
    assert fp["achieved"] == pytest.approx(bench.kernel_fp64_ops(m, n, nnz)[0] / 248.0e-6 / 1e9)
    # the slower kernel is the dominant one, whichever it is
    r2 = bench.roofline("powerlaw", m, n, nnz, [1.0, 2.0], [10, 10], {}, "float")
    assert r2["kernel"].startswith("dual_step_kernel<float>") and "fp64_alu" not in r2
    assert r2["algorithmic_bytes_per_launch"] == bench.kernel_bytes(m, n, nnz, 4)[1]


def test_peak_is_the_measured_copy_bandwidth():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak, kind = bench.measured_peaks()
    if os.path.exists(path):
        assert kind == "measured" and peak == float(json.load(open(path))["hbm_gbs"])
    else:
        assert (peak, kind) == (6800.0, "fallback")


def test_traffic_table_matches_the_byte_model_of_the_captured_instances():
    """Each recorded (traffic, algorithmic bytes) pair: the algorithmic bytes
    are kernel_bytes of the instance that was captured (transport at full
    size, the power-law recipe at scale 0.1), and the traffic is within
    [0.8, 1.1] of them (no re-reads)."""
    tr = bench.make_lp("transport")
    pl = bench.make_lp("powerlaw", 0.1)
    sizes = {"transport": (tr.m, tr.n, tr.nnz), "powerlaw": (pl.m, pl.n, pl.nnz)}
    for (kind, which, label), (traffic, alg, source) in bench.NCU_TRAFFIC.items():
        pb, db = bench.kernel_bytes(*sizes[kind], 4 if label == "float" else 8)
        assert alg == (pb if which == "primal" else db), (kind, which, label)
        assert 0.8 <= traffic / alg <= 1.1, (kind, which, label)
        assert os.path.exists(os.path.join(ROOT, source.split(" ")[0])), source


def test_median_rate_takes_the_median_step():
    runs = [(200.0, {"iterations": 640}, 0), (300.0, {"iterations": 640}, 0), (190.0, {"iterations": 640}, 0)]
    assert bench.median_rate(runs) == pytest.approx(640 / 0.2)
    assert bench.median_rate(runs[:1]) == pytest.approx(640 / 0.2)


def test_kernel_bytes_per_unit():
    """Per nonzero 12 bytes in FP64 (int32 index + double) and 8 in FP32 in
    each kernel; per primal row 4 (row pointer) + 8 vectors; per dual row
    4 + 8 vectors + 1 sense byte; one gathered vector each."""
    p1, d1 = bench.kernel_bytes(0, 0, 1, 8)
    assert (p1, d1) == (12, 12)
    assert bench.kernel_bytes(0, 0, 1, 4) == (8, 8)
    assert bench.kernel_bytes(0, 1, 0, 8) == (4 + 64, 8)
    assert bench.kernel_bytes(1, 0, 0, 8) == (8, 4 + 64 + 1)
