"""Host logic of bench.py that its JSON line rests on (CPU): the algorithmic
bytes of one half-sweep, the current-profile check behind `traffic`, the
measured peak, and the clock summary with its throttle reasons."""
import json
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1204_6192_gb300 import build, inputs  # noqa: E402


def _fake_ctx(W):
    return types.SimpleNamespace(W=W)


def test_algorithmic_bytes_of_the_bench_workload():
    # L = 128, 48 systems, FP16 spins (S = 6 B), FP16 couplings and field (2 B each).
    # Fused: per update 2 S + (3 bonds + 3 field) * 2 B / W; a half-sweep launch
    # updates N/2 sites x 48 systems: 1048576 * (2*6*48 + 12) = 616.6 MB.
    wl = inputs.workload("L128_fp16")
    assert bench.bytes_per_update(wl, 48) == pytest.approx(12.25)
    assert bench.algorithmic_half_sweep_bytes(_fake_ctx(48), wl) == 1048576 * 588 == 616562688
    # two-pass: (N/2) (3 S W + 9 J_b) = 1048576 * (3*6*48 + 9*2)
    assert bench.algorithmic_half_sweep_bytes(_fake_ctx(48), wl, fused=False) == 1048576 * 882


def test_algorithmic_bytes_fp32_and_batches():
    wl = inputs.workload("L128_fp32")
    assert bench.algorithmic_half_sweep_bytes(_fake_ctx(48), wl) == 1048576 * (2 * 12 * 48 + 6 * 4)
    assert bench.algorithmic_half_sweep_bytes(_fake_ctx(48), wl, fused=False) == \
        1048576 * (3 * 12 * 48 + 9 * 4)
    wl = inputs.workload("batch512_mixedL")
    sites = sum(s.L ** 3 for s in wl.samples) // 2
    assert bench.algorithmic_half_sweep_bytes(_fake_ctx(32), wl) == sites * (2 * 12 * 32 + 6 * 4)


def test_roofline_entry_fractions():
    wl = inputs.workload("L128_fp16")
    # half-sweep kernel in the step: (ms per OR launch, sweep kind, ms per half-sweep, ms per HB)
    rl = bench.roofline_entry(_fake_ctx(48), wl, (0.17634, "half", 0.17634, 0.33),
                              value_ns=0.004177, peak=6686.5, peak_kind="measured")
    # the kernel on the fused bytes: 616.6 MB / 0.17634 ms = 3.50 TB/s = 0.52 of 6686.5 GB/s
    assert rl["frac"] == pytest.approx(0.523, abs=2e-3)
    assert rl["half_sweep"]["frac_two_pass"] == pytest.approx(0.784, abs=2e-3)
    # the step: 12.25 B / 6686.5 GB/s = 1.832 ps against 4.177 ps
    assert rl["step_frac"] == pytest.approx(0.4386, abs=2e-3)
    # fused kernel: one launch moves a whole sweep's bytes (1.233 GB)
    rl = bench.roofline_entry(_fake_ctx(48), wl, (0.17634, "staged", 0.17634, 0.33),
                              value_ns=0.004177, peak=6686.5, peak_kind="measured")
    assert rl["frac"] == pytest.approx(0.523, abs=2e-3)
    assert rl["kernel"].startswith("k_staged_half")
    for kind in ("fused", "wave"):
        rl = bench.roofline_entry(_fake_ctx(48), wl, (0.30, kind, 0.176, 0.33), value_ns=0.0035,
                                  peak=6686.5, peak_kind="measured")
        assert rl["algorithmic_bytes_per_launch"] == 2 * 616562688
        assert rl["frac"] == pytest.approx(2 * 616562688 / 0.30e-3 / 1e9 / 6686.5, rel=1e-3)
        assert rl["half_sweep"]["frac"] == pytest.approx(0.524, abs=2e-3)


def test_launches_per_step():
    info = types.SimpleNamespace(variant=1, sweep_kernel=1, n_passes=1, n_samples=1, Wp=48)
    wl = inputs.workload("L128_fp16")        # 1 HB + 5 OR, 48 systems: energies and PT folded
    assert bench.launches_per_step(info, wl) == 12 + 2
    info.sweep_kernel = 2                    # two fused pairs, one half-sweep sweep with energies
    assert bench.launches_per_step(info, wl) == 2 + 4 + 2 + 2
    info.sweep_kernel = 3                    # one wave launch per OR sweep
    assert bench.launches_per_step(info, wl) == 2 + 5 + 2
    info.sweep_kernel = 4                    # staged: one launch per half-sweep
    assert bench.launches_per_step(info, wl) == 12 + 2
    info = types.SimpleNamespace(variant=1, sweep_kernel=1, n_passes=17, n_samples=512, Wp=32)
    assert bench.launches_per_step(info, inputs.workload("batch512_mixedL", steps=1)) == 17 * 12 + 3


def test_traffic_is_reported_only_for_the_profiled_source(monkeypatch):
    with open(os.path.join(ROOT, "profiles", "traffic.txt")) as f:
        rec = json.load(f)["or_half_sweep_fp16"]
    assert rec["dram_bytes_per_launch"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    monkeypatch.setattr(build, "source_hash", lambda: rec["source_hash"])
    assert bench.traffic_summary("or_half_sweep_fp16") == rec["dram_bytes_per_launch"]
    monkeypatch.setattr(build, "source_hash", lambda: "0" * 16)
    assert bench.traffic_summary("or_half_sweep_fp16") is None
    assert bench.traffic_summary("no_such_kernel") is None


def test_measured_peak_is_read_from_the_driver_file():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(p):
        pytest.skip("no measured peaks here")
    with open(p) as f:
        hbm = float(json.load(f)["hbm_gbs"])
    assert bench.measured_peak() == (hbm, "measured")


def test_clock_summary_median_and_reasons():
    cs = bench.ClockSampler(0)
    cs.samples = [
        ["0", "2070", "2070", "900", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["0", "2055", "2070", "1300", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
        ["0", "2070", "2070", "1100", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
    ]
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    cs.samples.append(["0", "1500", "2070", "1000", "0x8", "Active", "Not Active", "Not Active",
                       "Not Active"])
    assert "hw_slowdown" in cs.summary()["reasons"]
    assert bench.ClockSampler(0).summary()["reasons"] == ["unsampled"]


def test_whole_job_value_counts_every_rank():
    # 2 ranks, 10 ms for the slowest, 1e6 updates each: 10e6 ns / 2e6 updates
    assert bench.whole_job_value(10.0, 1_000_000, 2) == pytest.approx(5.0)
