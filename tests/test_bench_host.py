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
    # M-step; per CG step the operator's kernels (3) and update + direction (2)
    assert bench._launches_per_fit([10, 20], 3, 2) == 3 + (2 + 5 * 10) + (2 + 5 * 20)
    # each residual replacement adds the accurate residual (4 kernels) and, in
    # the graph, the direction again and two gates per run of CG steps (one
    # run per replacement and per round); each true-residual check the
    # accurate residual, the check and the loop gate
    assert (bench._launches_per_fit([10], 3, 2, n_rr=3, n_check=2, op_rr=4)
            == 3 + 2 + 5 * 10 + 3 * 4 + 2 * 6 + 3 * 1 + 2 * (3 + 2))
    # driven from the host loop there is no gate kernel
    assert bench._launches_per_fit([10], 3, 2, n_rr=0, n_check=2, op_rr=4, graph=False) == 3 + 2 + 5 * 10 + 2 * 5
    assert bench._launches_per_fit([], 3, 2) == 3
    # the graph's rotated loop: a first product before each entry into the CG
    # loop (per EM iteration, or per verification round)
    assert bench._launches_per_fit([10, 20], 3, 2, rotated=True) == 3 + (2 + 5 * 10) + (2 + 5 * 20) + 2
    # with replacement: per replacement the direction and the first product
    # again, and two gates per run of CG steps (replacements + rounds)
    assert (bench._launches_per_fit([10], 3, 2, n_rr=3, n_check=2, op_rr=4, rotated=True)
            == 3 + 2 + 5 * 10 + 3 * 4 + 2 * 6 + 2 + 3 * 2 + 2 * (3 + 2))
    assert (bench._launches_per_fit([10], 3, 2, n_rr=3, n_check=2, op_rr=4, graph=False, rotated=True)
            == 3 + 2 + 5 * 10 + 3 * 4 + 2 * 5)


def test_launch_count_matches_the_launch_list():
    """The launch list of a fit (host loop, BF16 two-pass) has, per CG step,
    two GEMMs, the T reduction, the update and the direction: 5 kernels."""
    per_step = bench._launches_per_fit([1], 3, 2) - bench._launches_per_fit([0], 3, 2)
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


def test_fp32_alu_peak_from_unit_counts_and_clock():
    # 152 SMs x 128 FP32 lanes x 2 flop per FMA x 2070 MHz
    assert bench._fp32_peak_tflops(2070) == pytest.approx(80.55, rel=1e-3)
    assert bench._fp32_peak_tflops(1035) == pytest.approx(bench._fp32_peak_tflops(2070) / 2)


def test_roofline_object_for_hbm_and_alu_bounds():
    # BF16 dense operator at 8192 x 32768, Q = 33: bytes over the measured copy peak
    alg_bytes = 2.0 * 8192 * 32768 * 2 + 2.0 * 33 * 32768 * 4
    r = bench._roofline({"bound": "hbm", "kernel": "k"}, 0.186, alg_bytes, None, 1093.6e6, 6795.1, "measured",
                        {"sm_mhz": 2070.0})
    assert r["unit"] == "GB/s" and r["peak"] == 6795.1 and r["traffic"] == 1093.6e6
    assert r["achieved"] == pytest.approx(alg_bytes / 0.186e-3 / 1e9) and r["frac"] == pytest.approx(r["achieved"] / 6795.1)
    # convolution operator (D = 1e6, L = 256, Q = 17): flops over the FP32 FMA peak at the sampled clock
    flops = 4.0 * 256 * 1e6 * 17
    a = bench._roofline({"bound": "alu", "kernel": "k"}, 0.427, 2.0 * 17 * 1e6 * 4, flops, None, 6795.1, "measured",
                        {"sm_mhz": 1980.0})
    assert a["unit"] == "TFLOP/s" and a["peak"] == pytest.approx(bench._fp32_peak_tflops(1980.0))
    assert a["achieved"] == pytest.approx(flops / 0.427e-3 / 1e12) and 0.0 < a["frac"] < 1.0
    assert "1980 MHz" in a["peak_source"]
    # no clock record: the maximum SM clock
    assert bench._roofline({"bound": "alu"}, 1.0, 0.0, 1e12, None, 1.0, "m", None)["peak"] == \
        pytest.approx(bench._fp32_peak_tflops(2070.0))


def test_profile_commands_use_existing_bench_flags():
    """Every `python bench.py ...` command quoted in profiles/*.md parses with
    the current command line of bench.py."""
    import glob
    import re
    import shlex
    cmds = []
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        text = open(path).read().replace("\\\n", " ")
        for m in re.finditer(r"python bench\.py([^\n`\"]*)", text):
            cmds.append((os.path.basename(path), m.group(1)))
    assert cmds
    for name, tail in cmds:
        argv = [a for a in shlex.split(tail) if not a.startswith("$")]
        bench._parser().parse_args(argv)   # raises SystemExit on an unknown flag
