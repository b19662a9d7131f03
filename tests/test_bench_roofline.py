"""The bench line's roofline arithmetic on CPU, from a made-up per-kind profile:
the dominant kind is the one with the most device time, `achieved` is its
algorithmic bytes over its summed event time, `traffic` scales the committed
DRAM-per-algorithmic-byte ratio to one launch, and the peaks are the measured
ones when the peaks file is present."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


def _prof():
    # 10 launches of 2 GB in 40 ms, 5 launches of 1 GB in 10 ms
    return {"guess_net": {"launches": 10, "total_ms": 40.0, "alg_bytes": 20e9},
            "gram": {"launches": 5, "total_ms": 10.0, "alg_bytes": 5e9}}


def test_dominant_kind_and_achieved_bandwidth(bench):
    r = bench.roofline_of("no_such_workload", _prof())
    assert r["kernel"] == "guess_net"
    assert r["achieved"] == pytest.approx(20e9 / 0.040 / 1e9)      # 500 GB/s
    assert r["alg_bytes_per_launch"] == pytest.approx(2e9)
    assert r["share_of_kernel_time"] == pytest.approx(0.8)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] is None                                     # no ratio file for this workload


def test_traffic_scales_the_committed_ratio_to_one_launch(bench):
    with open(os.path.join(ROOT, "profiles", "traffic_batched_scalar_1024.json")) as f:
        ratio = json.load(f)["guess_net"]["dram_per_alg_byte"]
    r = bench.roofline_of("batched_scalar_1024", _prof())
    assert r["traffic"] == pytest.approx(ratio * 2e9)


def test_peaks_are_the_measured_ones(bench):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(path):
        pytest.skip("no measured peaks on this machine")
    with open(path) as f:
        pk = json.load(f)
    hbm, src = bench._peak()
    assert (hbm, src) == (pk["hbm_gbs"], "measured")
    tf, tsrc = bench._tensor_peak()
    assert tf == pk["bf16_tflops_sustained"] and tsrc.startswith("measured")
