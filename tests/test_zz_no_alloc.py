"""The allocation-free mobility product (am_rpy_matvec_noalloc) for callers
that cannot allocate device memory, e.g. code running where cudaMalloc is not
allowed or not safe.  It must give what am_rpy_matvec gives with a caller
workspace, call after call (its scratch array is shared and keeps the last
call's contents), and refuse sizes beyond its fixed scratch.

Collected last on purpose (file name), so a run that stops at the first
failure has run every other test before this one."""
import numpy as np
import pytest

from paper_2107_10800_gb300 import build, binding, workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-5}  # the bars of the other mobility tests


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    build.build()
    binding.lib()
    return t


def with_workspace(torch, r, lam, wall, prec):
    dev = torch.device("cuda")
    n = len(r)
    dr, dl = torch.tensor(r, device=dev), torch.tensor(lam, device=dev)
    du = torch.empty_like(dr)
    nbytes = binding.rpy_matvec_workspace(n, prec)
    work = torch.empty(nbytes // 8 + 64, dtype=torch.float64, device=dev)
    aligned = (work.data_ptr() + 255) // 256 * 256
    binding.rpy_matvec_ptr(dr.data_ptr(), dl.data_ptr(), du.data_ptr(), n, 1.0, 0.1, wall, prec,
                           aligned, nbytes, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return du.cpu().numpy()


def without_alloc(torch, r, lam, wall, prec):
    dev = torch.device("cuda")
    n = len(r)
    dr, dl = torch.tensor(r, device=dev), torch.tensor(lam, device=dev)
    du = torch.full_like(dr, np.nan)
    binding.rpy_matvec_noalloc_ptr(dr.data_ptr(), dl.data_ptr(), du.data_ptr(), n, 1.0, 0.1, wall,
                                   prec, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return du.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("wall", [0, 1])
def test_noalloc_matches_workspace_version_twice(torch, prec, wall):
    # two calls in a row with different sizes and inputs: the second must
    # not see anything the first left in the shared scratch
    for seed, n in ((11, 3001), (12, 517)):
        r, lam = W.random_blobs(seed, n, a=0.1, wall=wall)
        ref = with_workspace(torch, r, lam, wall, prec)
        got = without_alloc(torch, r, lam, wall, prec)
        assert np.all(np.isfinite(got))
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= TOL[prec], (seed, n, err)
        # the same kernels with the same source split in the same order:
        # the two results agree bit for bit
        assert np.array_equal(got, ref), (seed, n, err)


def test_noalloc_rejects_sizes_beyond_scratch(torch):
    n = 200_000
    assert binding.rpy_matvec_workspace(n, "fp64") > binding.NOALLOC_SCRATCH_BYTES
    with pytest.raises(binding.AmError) as e:
        binding.rpy_matvec_noalloc_ptr(1, 1, 1, n, 1.0, 0.1, 0, "fp64", None)
    assert e.value.code == binding.AM_ERR_ARG
    assert "scratch" in str(e.value)
