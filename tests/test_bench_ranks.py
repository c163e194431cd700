"""The multi-GPU bench path on CPU: `bench.py --gpus N` runs one replica per
rank and reports the slowest rank's time with the work of all ranks.  Two
gloo ranks on this host check that aggregation, and that the reference arm
prints only on rank 0."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, w = bench.aggregate_ranks(dist, 100.0 + 50.0 * rank, 1e9 * (rank + 1), "cpu")
    out[rank] = (t, w)
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        assert res[r] == (150.0, 3e9)


def test_aggregate_without_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(None, 12.5, 7.0) == (12.5, 7.0)


def test_reference_arm_prints_on_rank_zero_only(tmp_path):
    """Under torchrun the reference arm runs on rank 0; other ranks exit 0
    without output (checked for rank 1 directly, no process group needed)."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
