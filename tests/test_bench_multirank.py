"""bench.py with more than one rank, on CPU (gloo, world size 2; no GPU).
The path has no data-path collective (replicas: one whole workload per
GPU), so what runs across ranks is the timing: every rank's time reduced to
the slowest one, and the reference arm printed by rank 0 alone while the
other ranks exit without work."""
import json
import os
import socket
import subprocess
import sys
from pathlib import Path

import pytest
import torch.multiprocessing as mp

ROOT = Path(__file__).resolve().parents[1]


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, values, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, str(ROOT))
    import torch.distributed as D
    import bench
    D.init_process_group("gloo", rank=rank, world_size=world)
    out[rank] = bench.max_over_ranks(values[rank], D, "cpu")
    D.barrier()
    D.destroy_process_group()


def test_time_is_the_slowest_ranks():
    values = [3.25, 7.5]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, _free_port(), values, out), nprocs=2, join=True)
        got = dict(out)
    assert got == {0: 7.5, 1: 7.5}


def test_single_process_keeps_its_value():
    sys.path.insert(0, str(ROOT))
    import bench
    assert bench.max_over_ranks(4.0, None, "cpu") == 4.0


def test_reference_arm_under_torchrun_prints_once():
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                        "--master-port", str(_free_port()), str(ROOT / "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-3000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
