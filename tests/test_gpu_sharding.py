"""The sharded product on the GPU with in-process shards: each shard's rows
of u = M lambda from am_rpy_matvec_rows (positions and forces of all shards
on the device), computed one after another on one GPU, reproduce the full
product and the oracle (free space and wall, FP64 and mixed)."""
import numpy as np
import pytest

from paper_2107_10800_gb300 import build, binding, sharding, workloads as W
from oracle import mobility as om
from oracle.system import System

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.lib()


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


@pytest.mark.parametrize("wall", [0, 1])
@pytest.mark.parametrize("n_ranks", [2, 3])
def test_shards_reproduce_the_full_product(wall, n_ranks):
    torch = pytest.importorskip("torch")
    w = W.chains_free_space(12) if not wall else W.diatom_colony(12, n_rods=8, nx=12)
    w = dict(w, assembly=np.arange(len(w["q"])))  # every body its own articulated body
    S = System(w)
    lam = np.random.default_rng(2).standard_normal((S.Nb, 3))
    plan = sharding.ShardPlan(w, n_ranks)
    r_all = S.r[plan.perm]
    lam_all = lam[plan.perm]
    ref = om.mobility_matvec(S.r, lam, w["a"], w["eta"], wall)[plan.perm]
    n = len(r_all)
    dr = torch.tensor(r_all, device="cuda")
    dl = torch.tensor(lam_all, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for prec, bar in (("fp64", 1e-12), ("mixed", 1e-5)):
        parts = []
        for k in range(n_ranks):
            row0, nrows = int(plan.blob0[k]), int(plan.nb[k])
            du = torch.empty((nrows, 3), dtype=torch.float64, device="cuda")
            nbytes = binding.rpy_matvec_rows_workspace(n, nrows, prec)
            work = torch.empty(nbytes // 8 + 64, dtype=torch.float64, device="cuda")
            wp = (work.data_ptr() + 255) // 256 * 256
            binding.rpy_matvec_rows_ptr(dr.data_ptr(), dl.data_ptr(), du.data_ptr(), n, row0, nrows,
                                        w["eta"], w["a"], wall, prec, wp, nbytes, stream)
            torch.cuda.synchronize()
            parts.append(du.cpu().numpy())
        assert rel(np.concatenate(parts), ref) <= bar


def test_rows_argument_checks():
    L = binding.lib()
    assert L.am_rpy_matvec_rows(None, None, None, 10, 5, 6, 1.0, 0.1, 0, 0, None, 0, None) == binding.AM_ERR_ARG
    assert L.am_rpy_matvec_rows(None, None, None, 10, -1, 2, 1.0, 0.1, 0, 0, None, 0, None) == binding.AM_ERR_ARG
    assert L.am_rpy_matvec_rows(None, None, None, 10, 3, 0, 1.0, 0.1, 0, 0, None, 0, None) == binding.AM_OK
