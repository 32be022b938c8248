"""Host logic of bench.py's roofline lines (no GPU): the algorithmic work per launch over its
duration against the peak, the larger of the FP32 and MUFU fractions for the ALU-bound kernels, and
the ncu DRAM figures attached only to the workload they were captured at."""
import pytest

import bench

PEAKS = {"hbm_gbs": 6000.0, "fp32_tops": 40.0, "mufu_tops": 10.0}
STATS = {"n_hits": 1_000_000, "n_composited": 900_000, "n_replayed": 900_000, "n_pairs": 2_000_000,
         "n_visible": 50_000}


def test_alu_roofline_takes_the_larger_fraction():
    r = bench.roofline_of("replay_bwd", 2.0, STATS, 0, PEAKS, "measured")
    ops = STATS["n_replayed"] * bench.OPS_REPLAY
    mufu = STATS["n_replayed"] * bench.MUFU_REPLAY
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(ops / 2e-3 / 1e12)
    assert r["fp32_frac"] == pytest.approx(ops / 2e-3 / 1e12 / PEAKS["fp32_tops"])
    assert r["mufu_frac"] == pytest.approx(mufu / 2e-3 / 1e12 / PEAKS["mufu_tops"])
    assert r["frac"] == max(r["fp32_frac"], r["mufu_frac"])


def test_hbm_roofline_counts_the_algorithmic_bytes():
    r = bench.roofline_of("bin_emit", 0.5, STATS, 0, PEAKS, "measured")
    b = STATS["n_pairs"] * 12 + STATS["n_visible"] * 160
    assert r["bound"] == "hbm" and r["algorithmic_bytes"] == b
    assert r["achieved"] == pytest.approx(b / 0.5e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / PEAKS["hbm_gbs"])


@pytest.mark.parametrize("phase", ["composite", "replay_bwd", "sort", "bin_emit"])
def test_dram_figures_only_at_their_workload(phase):
    # another workload (the batched step, a reduced case): never the full-size render's figure
    assert bench.roofline_of(phase, 1.0, STATS, 0, PEAKS, "measured")["traffic"] is None
    # the render workload: the recorded figure while the kernel sources hash to its fingerprint
    got = bench.roofline_of(phase, 1.0, STATS, 0, PEAKS, "measured", True)["traffic"]
    assert got is None or got == bench.MEASURED_TRAFFIC[phase][0]
    assert got == bench._traffic(phase)
