"""Multi-rank plumbing of bench.py on CPU (gloo, world size 2): process-group set-up
from the torchrun environment, the barrier, the max-over-ranks time and the
whole-job sums, and the reference arm's rule that only rank 0 runs and prints.
The benchmarked path runs independent replicas with no data-path collective, so
these are the only multi-rank pieces.
"""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, outdir):
    os.environ.update(WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import contextlib
    import io
    import types

    import torch.distributed as dist

    import bench

    world, r, local = bench.dist_setup()
    bench.barrier(world)
    mx = bench.allreduce_max(world, 3.0 * (rank + 1))
    sm = bench.allreduce_sum(world, float(rank + 1))
    buf = io.StringIO()
    if rank == 1:
        args = types.SimpleNamespace(edge=16, nmol=4, steps=2, warmup=1, gpus=2)
        with contextlib.redirect_stdout(buf):
            bench.run_reference(args, world, rank)
    backend = dist.get_backend()
    bench.barrier(world)
    dist.destroy_process_group()
    with open(os.path.join(outdir, f"r{rank}.json"), "w") as f:
        json.dump({"world": world, "rank": r, "max": mx, "sum": sm, "printed": buf.getvalue(),
                   "backend": backend}, f)


def test_two_rank_gloo_plumbing(tmp_path):
    import torch
    import torch.multiprocessing as mp
    if torch.cuda.is_available():
        pytest.skip("checks the CPU (gloo) path")
    mp.spawn(_worker, args=(_free_port(), str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for r, d in enumerate(res):
        assert d["world"] == 2 and d["rank"] == r and d["backend"] == "gloo"
        assert d["max"] == 6.0 and d["sum"] == 3.0
    assert res[1]["printed"] == ""
