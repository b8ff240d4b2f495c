"""The multi-rank path of bench.py on CPU: two processes over gloo.  Each
rank runs its own replica of the workload (the sweep has no data-path
exchange); the job's time is the slowest rank's (one MAX all-reduce) and
its throughput is every rank's units over that time."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    dist.barrier()
    slowest = bench.max_over_ranks(1.5 + rank, ws, device="cpu")
    value = bench.job_value(ws, 1000 * (rank + 1), slowest)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{slowest} {value}\n")


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = root + os.pathsep + os.environ.get("PYTHONPATH", "")
    import sys
    if root not in sys.path:
        sys.path.insert(0, root)
    ws, port = 2, _free_port()
    mp.spawn(_rank_main, args=(ws, port, str(tmp_path)), nprocs=ws, join=True)
    got = [tuple(map(float, open(tmp_path / f"rank{r}.txt").read().split())) for r in range(ws)]
    for slowest, value in got:
        assert slowest == 2.5  # rank 1's time
    # every rank computes the job value from its own units; rank 0 prints it
    assert got[0][1] == ws * 1000 / 2.5
