"""The multi-rank path of bench.py on CPU: two gloo ranks (the GPU runs use
one process per GPU over NCCL with the same calls).  Each rank times its own
suspension; the whole-job figures take the slowest rank's time and all
ranks' pairs."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2107_10800_gb300 import workloads as W
    # rank r: 2 + r seconds, 1000 (r + 1) pairs, end-to-end step 10 (r + 1) ms
    res = bench.combine_ranks(torch, 2.0 + rank, 1000 * (rank + 1), 10.0 * (rank + 1), 4, "cpu")
    w = bench.rank_workload(W, rank)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, res, float(w["q"][0, 2])))


def test_two_ranks_combine_max_time_and_summed_pairs():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict()
    for _ in range(world):
        rank, res, z0 = q.get(timeout=120)
        got[rank] = (res, z0)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(world):
        secs, pairs, e2e = got[rank][0]
        assert secs == 3.0            # the slowest rank's timed region
        assert pairs == 3000.0        # every rank's pairs
        assert e2e == pytest.approx(3000.0 / 4 / 0.020)
    # the ranks run different (independent) suspensions
    assert got[0][1] != got[1][1]
