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
                split_slice_pairs=0, gemm_launches=0, tc_launches=0, split_launches=0, fp64_bytes=0.0,
                tc_bytes=0.0, split_bytes=0.0)
    base.update(kw)
    return SimpleNamespace(**base)


def test_hbm_bound_below_the_ridge_point():
    """1e5 stored 64 x 64 pairs (5.2e10 flops) and 1e10 algorithmic bytes in
    10 ms on the TF32 kernel: 5.2 flop/byte, far below the TF32 ridge
    (~140 flop/byte), so HBM binds and achieved = bytes / time."""
    bs = 64
    reps = [_rep(tc_ms=10.0, tc_pairs=10 ** 5, tc_launches=28, tc_bytes=1e10)]
    k = bench.kernel_rooflines(reps, bs, "tf32")["tc"]
    hbm, _ = bench.hbm_peak_gbs()
    assert k["bound"] == "hbm" and k["unit"] == "GB/s"
    assert k["achieved"] == pytest.approx(1e10 / 10e-3 / 1e9)
    assert k["frac"] == pytest.approx(k["achieved"] / hbm) == pytest.approx(k["hbm_frac"])
    flops = 1e5 * 2 * bs ** 3
    assert k["tflops"] == pytest.approx(flops / 10e-3 / 1e12)
    peak, _ = bench.tensor_peak_tflops("tf32")
    assert k["compute_frac"] == pytest.approx(k["tflops"] / peak)
    assert k["intensity_flop_per_byte"] == pytest.approx(flops / 1e10)
    assert k["algorithmic_bytes_per_launch"] == pytest.approx(1e10 / 28)
    assert k["avg_launch_us"] == pytest.approx(1e4 / 28)
    assert k["traffic"] is None and "traffic_source" not in k


def test_compute_bound_above_the_ridge_point():
    """A dense-like product: 1e6 pairs over 1e9 bytes (524 flop/byte) is
    above the BF16 ridge (~284 flop/byte): the tensor peak binds."""
    bs = 64
    reps = [_rep(tc_ms=1.0, tc_pairs=10 ** 6, tc_launches=1, tc_bytes=1e9)]
    k = bench.kernel_rooflines(reps, bs, "bf16")["tc"]
    peak, _ = bench.tensor_peak_tflops("bf16")
    want = 1e6 * 2 * bs ** 3 / 1e-3 / 1e12
    assert k["bound"] == "tensor" and k["unit"] == "TFLOP/s"
    assert k["achieved"] == pytest.approx(want) and k["frac"] == pytest.approx(want / peak)


def test_split_counts_its_slice_products():
    bs = 64
    # 100 stored pairs, each formed from 28 slice pairs, in 1 ms; FP64 pipe kernel beside it
    reps = [_rep(split_ms=1.0, split_pairs=100, split_slice_pairs=2800, split_launches=1, split_bytes=1e8,
                 gemm_ms=2.0, fp64_pairs=1000, gemm_launches=2, fp64_bytes=1e6)]
    k = bench.kernel_rooflines(reps, bs, "tf32")
    s = k["split"]
    assert s["fp64_equivalent_tflops"] == pytest.approx(100 * 2 * bs ** 3 / 1e-3 / 1e12)
    assert s["tflops"] == s["bf16_slice_tflops"] == pytest.approx(2800 * 2 * bs ** 3 / 1e-3 / 1e12)
    assert s["slice_pairs_per_block_pair"] == pytest.approx(28.0)
    # 1.47e9 slice flops over 1e8 bytes: 14.7 flop/byte, below the BF16 ridge (~284)
    assert s["bound"] == "hbm" and s["achieved"] == pytest.approx(1e8 / 1e-3 / 1e9)
    # a hundred times fewer bytes (1468 flop/byte): the BF16 peak binds the slice products
    reps[0].split_bytes = 1e6
    s = bench.kernel_rooflines(reps, bs, "tf32")["split"]
    peak, _ = bench.tensor_peak_tflops("bf16")
    assert s["bound"] == "tensor" and s["achieved"] == pytest.approx(s["bf16_slice_tflops"])
    assert s["frac"] == pytest.approx(s["bf16_slice_tflops"] / peak)
    f = k["fp64"]  # 1.05e9 flops over 1e6 bytes: far above the FP64 ridge (~0.16)
    assert f["bound"] == "alu" and f["achieved"] == pytest.approx(1000 * 2 * bs ** 3 / 2e-3 / 1e12)


def test_traffic_per_launch_from_the_capture():
    t65 = {"tc": (1.0e8, "capture")}
    reps = [_rep(tc_ms=10.0, tc_pairs=1000, tc_launches=28, tc_bytes=28 * 0.8e8, split_ms=20.0, split_pairs=100,
                 split_slice_pairs=2300, split_launches=8, split_bytes=1e9)]
    k = bench.kernel_rooflines(reps, 64, "tf32", t65)
    assert k["tc"]["traffic"] == 1.0e8 and k["split"]["traffic"] is None
    assert k["tc"]["traffic_unit"] == "bytes per launch" and "traffic_source" not in k["split"]
    assert k["tc"]["traffic_over_algorithmic"] == pytest.approx(1.25)


def test_traffic_table_names_existing_workloads():
    for name, table in bench.DRAM_TRAFFIC.items():
        assert name in bench.WORKLOADS
        assert bench.WORKLOADS[name]["prec"] == "tf32"  # the capture ran TF32 sweeps and split delta
        assert set(table) <= {"tc", "split", "fp64"}
        for key, (v, src) in table.items():
            assert v > 0 and "ncu capture" in src
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


def test_cpu_baseline_reports_both_thread_counts_and_the_exponent(oracle_mod):
    """The CPU anchor on the 4096-row chain (bs 32): all-core value measured
    on the workload itself, single-threaded value and the cost exponent
    measured at n = 2048 and 4096 (about linear for the banded chain)."""
    w = bench.WORKLOADS["irsi-chain-n4096-bs32"]
    assert bench.cpu_sizes(w) == (2048, 4096)
    c = bench.cpu_baseline(w)
    assert c["kind"] == "oracle" and c["cores"] == bench.nproc() and c["value"] > 0
    assert "measured on the workload itself" in c["sample"]
    st = c["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0 and set(st["seconds_at"]) == {"2048", "4096"}
    assert 0.5 < st["cost_exponent"] < 1.7
    assert bench.cpu_sizes(bench.WORKLOADS[bench.DEFAULT_WORKLOAD]) == (16384, 65536)
