"""The multi-process path of the benchmark on CPU (gloo, world size 2).

The method's single problem is not sharded (replicas only): under torchrun every
rank solves its own problem and the ranks exchange one scalar, the largest
time.  These tests run that exchange and the reference arm's rank gating in two
CPU processes."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + 2.0 * rank, "cpu", world)     # rank times 1 s and 3 s
    rate = bench.job_rate(1000, 5, world, t)
    dist.barrier()
    dist.destroy_process_group()
    with open(out + f".{rank}", "w") as fh:
        json.dump({"max": t, "rate": rate}, fh)


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_max_over_ranks_and_job_rate_gloo(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "res")
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        with open(out + f".{r}") as fh:
            d = json.load(fh)
        assert d["max"] == 3.0                       # the slowest rank's time on every rank
        assert d["rate"] == pytest.approx(2 * 1000 * 5 / 3.0)   # all ranks' units over that time


def test_reference_arm_prints_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, cwd=ROOT, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--M", "1024", "--N", "4096"], capture_output=True, text=True, env=env,
                       cwd=ROOT, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
