"""Host-side pieces of bench.py (no GPU): the algorithmic FLOP count and peak
of the tensor-core roofline, the figures read from the committed ncu summary,
and the reference arm's JSON line (the FP64 oracle on the host cores)."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tensor_flops_count_three_products_of_the_contraction():
    # P = A W with A one row of 2K+1 harmonics and W (2K+1) x (4K+1): 2 (2K+1)(4K+1) FLOP, three times
    assert bench.tensor_flops_per_step(10) == 3 * 2 * 21 * 41 == 5166
    assert bench.tensor_flops_per_step(4) == 3 * 2 * 9 * 17


def test_method_work_is_the_direct_sum_count():
    # 8 FMAs per half-mode (H = 220 at K = 10) + ~90 per step, 2 FLOP per FMA
    assert bench.method_flops_per_step(10) == 2 * (8 * 220 + 90) == 3700
    assert bench.method_flops_per_step(2) == 2 * (8 * 12 + 90)


def test_tensor_roofline_counts_the_method_work_against_the_operand_peak():
    # the headline workload: 1.75e9 particle-steps in 26.717 ms on FP16 operands
    r = bench.tensor_roofline(10, 1_750_000_000, 26.717, {"bf16_tflops": 1936.3}, "measured")
    assert r["bound"] == "tensor" and r["peak"] == 1936.3
    assert abs(r["achieved"] - 1.75e9 * 3700 / 26.717e-3 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 1936.3) < 1e-12
    assert abs(r["frac"] - 0.1252) < 1e-3
    assert abs(r["tensor_issued_frac"] - 1.75e9 * 5166 / 26.717e-3 / 1e12 / 1936.3) < 1e-12


def test_fp32_roofline_counts_the_executed_fmas_against_the_fp32_pipe():
    r = bench.fp32_roofline(10, 1_750_000_000, 64.4, {"sm_max_mhz": 2070.0}, "measured", 152)
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    assert abs(r["peak"] - peak) < 1e-9
    assert abs(r["frac"] - 1.75e9 * 1840 / 64.4e-3 / 1e12 / peak) < 1e-12
    assert abs(r["frac"] - 0.621) < 2e-3
    assert r["method_work_frac"] > 1.0  # the product basis does half the direct sum's work


def test_peak_follows_the_operand_type():
    peaks = {"bf16_tflops": 1898.6}
    assert bench.tensor_operands(10) == "f16" and bench.tensor_operands(8) == "tf32"
    assert bench.tensor_peak(10, peaks, "measured")[0] == 1898.6
    assert abs(bench.tensor_peak(8, peaks, "measured")[0] - 1898.6 * 1.1 / 2.25) < 1e-9


def test_committed_profile_figures_are_read():
    traffic = bench.profile_traffic("timedep_k10_tc_kernel.md")
    issue = bench.profile_value("timedep_k10_tc_kernel.md", "issue_active_frac")
    assert isinstance(traffic, int) and traffic > 0
    assert 0.0 < issue <= 1.0
    assert bench.profile_value("timedep_k10_tc_kernel.md", "no_such_key") is None


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["unit"] == "particle-steps/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
