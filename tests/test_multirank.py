"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the timed
region is the maximum over ranks, each rank gets an independent problem (weak
scaling, no data-path collective), and under torchrun the reference arm runs on
rank 0 only and prints exactly one JSON line."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ms_per_rank, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench._aggregate_over_ranks(ms_per_rank[rank], world, dist, torch.device("cpu"))
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"t_max": t}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_timed_region_is_max_over_two_gloo_ranks(tmp_path):
    ms = [12.5, 40.25]
    mp.spawn(_rank_main, args=(2, _free_port(), ms, str(tmp_path)), nprocs=2, join=True)
    got = [json.load(open(tmp_path / f"r{r}.json"))["t_max"] for r in range(2)]
    assert got == [max(ms), max(ms)]


def test_single_rank_aggregation_needs_no_process_group():
    import bench
    assert bench._aggregate_over_ranks(7.0, 1) == 7.0


def test_ranks_get_independent_problems():
    from synth import workload
    a, _ = workload("dense_n256_d1024_k20", seed=1)
    b, _ = workload("dense_n256_d1024_k20", seed=2)
    assert a.phi.shape == b.phi.shape and not np.array_equal(a.phi, b.phi)
    assert not np.array_equal(a.z, b.z)


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--workload", "dense_n256_d1024_k20", "--cpu-budget", "2"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
