"""The benchmark's multi-rank host logic on CPU, world size 2 over gloo (the
path is replicas only: one independent apply per rank, no data-path
collective):

* the timed per-step time is the maximum over ranks, and the reported rate
  counts the units of all ranks (whole-job throughput);
* the reference arm under torchrun runs on rank 0 alone and prints exactly
  one JSON line; the other rank exits 0 without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_job(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms, rate = bench.job_time_and_rate([1.5, 4.0][rank], 1000, world)
    with open(f"{out}.{rank}", "w") as fh:
        json.dump([ms, rate], fh)
    dist.destroy_process_group()


def test_job_time_is_the_max_over_two_gloo_ranks(tmp_path):
    out = str(tmp_path / "rank")
    mp.start_processes(_rank_job, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    for r in range(2):
        with open(f"{out}.{r}") as fh:
            ms, rate = json.load(fh)
        assert ms == 4.0
        assert rate == pytest.approx(2 * 1000 / 4.0e-3)


def test_single_rank_needs_no_process_group():
    import bench

    ms, rate = bench.job_time_and_rate(2.0, 500, 1)
    assert ms == 2.0 and rate == pytest.approx(500 / 2.0e-3)


def test_reference_arm_under_two_ranks_prints_one_line():
    env = dict(os.environ, OMP_NUM_THREADS=str(os.cpu_count() or 1))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
