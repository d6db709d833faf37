"""Host-side pieces of bench.py that need no GPU: the kernel-launch count it
reports, the NMSE, the metric name and the roofline denominators."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from synth import WORKLOADS  # noqa: E402


def test_launch_count_per_fit():
    # 3 per fit (b, finiteness check of y, set-up); per EM iteration init and
    # M-step; per CG step the operator's kernels and update + direction
    assert bench._launches_per_fit([10, 20], 0, 3, 4, 2) == 3 + (2 + 5 * 10) + (2 + 5 * 20)
    # a residual replacement every 3 steps adds the operator on X and the residual kernel
    assert bench._launches_per_fit([10], 3, 3, 4, 2) == 3 + 2 + 5 * 10 + 3 * (4 + 1)
    assert bench._launches_per_fit([], 0, 3, 4, 2) == 3


def test_launch_count_matches_the_launch_list():
    """The launch list of a fit (host loop, BF16 two-pass) has, per CG step,
    two GEMMs, the T reduction, the update and the direction: 5 kernels."""
    per_step = bench._launches_per_fit([1], 0, 3, 4, 2) - bench._launches_per_fit([0], 0, 3, 4, 2)
    assert per_step == 5


def test_nmse_db():
    z = np.array([3.0, -4.0, 0.0])
    assert bench._nmse_db(1.1 * z, z) == pytest.approx(-20.0)
    assert bench._nmse_db(z, z) < -3000.0   # exact: floored, not -inf


def test_metric_name_names_the_workload():
    name = bench._metric_name("dense_n8192_d32768_k32_bf16", WORKLOADS["dense_n8192_d32768_k32_bf16"])
    assert name == "CoFEM EM-iter/s (dense N=8192 D=32768, K=32, T=30, BF16 Phi)"
    conv = bench._metric_name("toeplitz_d1e6_l256_k16", WORKLOADS["toeplitz_d1e6_l256_k16"])
    assert "convolutional N=D=1000000 L=256" in conv


def test_peaks_come_from_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._peaks() == (6800.0, 1900.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6795.1, "bf16_tflops": 1846.0}))
    assert bench._peaks() == (6795.1, 1846.0, "measured")
