"""Host-side arithmetic of bench.py (no GPU): achieved rates from
block-pair counts and CUDA-event times, fractions of the peak, the DRAM
traffic figures taken from an ncu capture, and the clock samples of the
timed region."""
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _rep(**kw):
    base = dict(gemm_ms=0.0, tc_ms=0.0, split_ms=0.0, fp64_pairs=0, tc_pairs=0, split_pairs=0,
                split_slice_pairs=0, gemm_launches=0, tc_launches=0, split_launches=0)
    base.update(kw)
    return SimpleNamespace(**base)


def test_achieved_and_fraction_from_pairs_and_time():
    bs = 64
    # 1e6 stored pairs of 64 x 64 blocks in 10 ms on the TF32 kernel, 28 launches
    reps = [_rep(tc_ms=10.0, tc_pairs=10 ** 6, tc_launches=28)]
    k = bench.kernel_rooflines(reps, bs, "tf32")
    want = 1e6 * 2 * bs ** 3 / 10e-3 / 1e12
    assert k["tc"]["achieved"] == pytest.approx(want)
    peak, _ = bench.tensor_peak_tflops("tf32")
    assert k["tc"]["frac"] == pytest.approx(want / peak)
    assert k["tc"]["avg_launch_us"] == pytest.approx(1e4 / 28)
    assert k["tc"]["traffic"] is None and "traffic_source" not in k["tc"]
    assert "fp64" not in k and "split" not in k


def test_split_rate_counts_slice_pairs():
    bs = 64
    # 100 stored pairs, each formed from 28 slice pairs, in 1 ms
    reps = [_rep(split_ms=1.0, split_pairs=100, split_slice_pairs=2800, split_launches=1)]
    k = bench.kernel_rooflines(reps, bs, "tf32")["split"]
    assert k["achieved"] == pytest.approx(2800 * 2 * bs ** 3 / 1e-3 / 1e12)
    assert k["fp64_equivalent_tflops"] == pytest.approx(100 * 2 * bs ** 3 / 1e-3 / 1e12)
    assert k["slice_pairs_per_block_pair"] == pytest.approx(28.0)


def test_traffic_per_launch_from_the_capture():
    t65 = bench.DRAM_TRAFFIC["irsi-mixed-chain-n65536-bs64"]
    t262 = bench.DRAM_TRAFFIC["irsi-mixed-chain-n262144-bs64"]
    assert t262["tc"][0] == pytest.approx(4 * t65["tc"][0])
    # the per-launch average of the captured factorization's 28 TF32 launches
    assert t65["tc"][0] == pytest.approx(168.35e6, rel=1e-3)
    # the split launches changed after the capture: no traffic figure
    assert "split" not in t65 and "split" not in t262
    reps = [_rep(tc_ms=10.0, tc_pairs=1000, tc_launches=28, split_ms=20.0, split_pairs=100,
                 split_slice_pairs=2300, split_launches=8)]
    k = bench.kernel_rooflines(reps, 64, "tf32", t262)
    assert k["tc"]["traffic"] == t262["tc"][0] and k["split"]["traffic"] is None
    assert k["tc"]["traffic_unit"] == "bytes per launch" and "traffic_source" not in k["split"]
    assert "65,536" in k["tc"]["traffic_source"]


def test_traffic_table_names_existing_workloads():
    for name, table in bench.DRAM_TRAFFIC.items():
        assert name in bench.WORKLOADS
        assert bench.WORKLOADS[name]["prec"] == "tf32"  # the capture ran TF32 sweeps and split delta
        assert set(table) <= {"tc", "split", "fp64"}
    assert bench.DEFAULT_WORKLOAD in bench.DRAM_TRAFFIC


def test_clock_summary_parses_samples_and_reasons(tmp_path):
    """The nvidia-smi sample file of the timed region: median SM clock, the
    largest max clock, and every throttle reason seen Active."""
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    rows = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",  # skipped
    ]
    with open(s.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    s.proc = object()  # as if sampling ran
    c = s.summary()
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s.proc = None
    assert s.summary() is None
