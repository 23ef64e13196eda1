"""One suspension sharded over several GPUs, one process per GPU: the
partitioning logic and the gather-then-local-rows mobility product.

Partition: whole articulated bodies go to ranks (largest first, each to the
rank with the fewest blobs so far), so that K, C, the links and the
block-diagonal preconditioner of Sec. 3.1 stay local to a rank.  The blobs
are renumbered rank by rank (within a rank in body order), so rank k owns
the contiguous rows blob0[k] .. blob0[k] + nb[k] - 1 of the product.

Product u = M lambda (Eq. RPY), per call: gather the positions and the
forces of all ranks (32 bytes per blob each way in FP64 of r and lambda; the
positions change once per step, the forces every GMRES iteration), then the
rank's own rows against all sources (am_rpy_matvec_rows).  A sharded GMRES
also needs a sum over ranks of its dot products (m + 1 scalars per Arnoldi
step); the library's single-GPU solver does not take that step.
"""
import numpy as np


def partition_assemblies(blobs_per_assembly, n_ranks):
    """Rank of every articulated body: largest first (ties: lower index), each
    to the rank with the fewest blobs so far (ties: lower rank)."""
    sizes = np.asarray(blobs_per_assembly, dtype=np.int64)
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(sizes)), key=lambda a: (-int(sizes[a]), a))
    load = np.zeros(n_ranks, dtype=np.int64)
    rank = np.zeros(len(sizes), dtype=np.int64)
    for a in order:
        k = int(np.argmin(load))  # first minimum: the lowest rank
        rank[a] = k
        load[k] += sizes[a]
    return rank


class ShardPlan:
    """Blob layout of a workload (the dict of workloads.py) sharded over
    n_ranks: perm[new] = old blob index, blob0[k], nb[k] the rows of rank k,
    bodies[k] the bodies of rank k (in body order)."""

    def __init__(self, w, n_ranks):
        off = np.asarray(w["blob_offset"], dtype=np.int64)
        asm = np.asarray(w["assembly"], dtype=np.int64)
        nblob = np.diff(off)
        n_asm = int(asm.max()) + 1
        per_asm = np.bincount(asm, weights=nblob, minlength=n_asm).astype(np.int64)
        self.rank_of_assembly = partition_assemblies(per_asm, n_ranks)
        rank_of_body = self.rank_of_assembly[asm]
        self.n_ranks = n_ranks
        self.bodies = [np.nonzero(rank_of_body == k)[0] for k in range(n_ranks)]
        perm, blob0, nb = [], [], []
        for k in range(n_ranks):
            blob0.append(len(perm))
            for p in self.bodies[k]:
                perm.extend(range(off[p], off[p + 1]))
            nb.append(len(perm) - blob0[-1])
        self.perm = np.asarray(perm, dtype=np.int64)
        self.blob0 = np.asarray(blob0, dtype=np.int64)
        self.nb = np.asarray(nb, dtype=np.int64)

    def local(self, rank, values):
        """The rows of `values` (per blob, old order) that rank owns."""
        v = np.asarray(values)
        return v[self.perm[self.blob0[rank]:self.blob0[rank] + self.nb[rank]]]


def sharded_mobility(plan, rank, r_local, lam_local, allgather, rows_product):
    """u for the blobs of `rank` (its rows, new order): gather r and lambda
    of all ranks (allgather(x) returns the ranks' arrays concatenated in rank
    order), then rows_product(r_all, lam_all, row0, nrows)."""
    r_all = allgather(np.asarray(r_local, float))
    lam_all = allgather(np.asarray(lam_local, float))
    return rows_product(r_all, lam_all, int(plan.blob0[rank]), int(plan.nb[rank]))


def torch_allgather(plan, group=None):
    """An allgather for sharded_mobility over torch.distributed (gloo on CPU
    tensors, NCCL on device tensors): pads every rank's rows to the largest
    count, gathers, and drops the padding."""
    import torch
    import torch.distributed as dist
    counts = [int(c) for c in plan.nb]
    width = max(counts) if counts else 0

    def gather(x):
        t = torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64)
        pad = torch.zeros((width,) + tuple(t.shape[1:]), dtype=t.dtype)
        pad[:t.shape[0]] = t
        parts = [torch.empty_like(pad) for _ in counts]
        dist.all_gather(parts, pad, group=group)
        return np.concatenate([p[:c].numpy() for p, c in zip(parts, counts)])
    return gather
