"""The N > 1 paths of the benchmark on CPU with world_size 2 (gloo), no GPU: the max-over-ranks
timing of replicas, and the reference arm under torchrun (rank 0 alone runs and prints)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = [120.0, 180.0][rank]                     # rank 1 is the slow replica
    out[rank] = bench.job_seconds_per_step(ms, steps=3, world=world, device="cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks():
    """Every rank gets the slowest rank's time, and s/step counts the steps of all replicas."""
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    for r in range(2):
        ms, sps = out[r]
        assert ms == 180.0
        assert abs(sps - 180.0 / 1e3 / (3 * 2)) < 1e-15


def test_reference_arm_under_torchrun():
    """`torchrun --nproc-per-node 2 bench.py --impl reference`: rank 0 prints one JSON line with
    n_gpus = 2, the other rank exits 0 without output."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
