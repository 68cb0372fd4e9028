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
