"""The sharding logic of one suspension over several processes, on CPU: the
partition keeps articulated bodies whole and balances blobs, the plan is a
permutation of the blobs, and two gloo ranks running the gather-then-rows
product (with the oracle's mobility rows as the local step) reproduce the
full product."""
import os
import socket
import sys

import numpy as np
import pytest

from paper_2107_10800_gb300 import sharding, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_partition_balanced_and_deterministic():
    rng = np.random.default_rng(0)
    sizes = rng.integers(1, 200, 57)
    for n_ranks in (1, 2, 3, 8):
        rank = sharding.partition_assemblies(sizes, n_ranks)
        assert np.array_equal(rank, sharding.partition_assemblies(sizes, n_ranks))
        load = np.bincount(rank, weights=sizes, minlength=n_ranks)
        assert load.sum() == sizes.sum()
        assert load.max() - load.min() <= sizes.max()


def test_plan_is_a_permutation_of_whole_assemblies():
    w = W.batched_chains(3, n_systems=1, lo=800, hi=1200)[0]
    plan = sharding.ShardPlan(w, 3)
    assert np.array_equal(np.sort(plan.perm), np.arange(w["blob_offset"][-1]))
    asm = np.asarray(w["assembly"])
    for k in range(3):
        owned = set(asm[plan.bodies[k]])
        for j in range(3):
            if j != k:
                assert owned.isdisjoint(asm[plan.bodies[j]])
    assert plan.nb.sum() == w["blob_offset"][-1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from oracle.mobility import mobility_rows
    from paper_2107_10800_gb300 import sharding as sh, workloads as Wk
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = Wk.chains_free_space(11)
    from oracle.system import System
    S = System(w)
    lam = np.random.default_rng(1).standard_normal((S.Nb, 3))
    plan = sh.ShardPlan(w, world)

    def rows(r_all, lam_all, row0, nrows):
        return mobility_rows(r_all, lam_all, np.arange(row0, row0 + nrows), w["a"], w["eta"], w["wall"])

    u = sh.sharded_mobility(plan, rank, plan.local(rank, S.r), plan.local(rank, lam), sh.torch_allgather(plan),
                            rows)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, u))


def test_two_gloo_ranks_reproduce_the_full_product():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    from oracle.mobility import mobility_matvec
    from oracle.system import System
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        rank, u = q.get(timeout=180)
        got[rank] = u
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = W.chains_free_space(11)
    S = System(w)
    lam = np.random.default_rng(1).standard_normal((S.Nb, 3))
    plan = sharding.ShardPlan(w, world)
    full = mobility_matvec(S.r, lam, w["a"], w["eta"], w["wall"])
    u = np.concatenate([got[0], got[1]])
    assert np.abs(u - full[plan.perm]).max() <= 1e-13 * np.abs(full).max()
