"""The symmetric FP64 all-pairs product (each unordered pair evaluated once
and applied in both directions, M_ji = M_ij^T; rpy_sym_f64 in csrc/rpy.cu)
through the C ABI, forced on every tile size: against the oracle's product
at the FP64 bar (1e-12, max-abs over max-abs) and against the one-direction
kernel, on sizes that leave ragged tiles, free space and above a wall; and a
batched FP64 solve on the symmetric layout, whose systems stop at different
iterations (stopped systems write zero partial sums), against the oracle's
dense solves at 1e-10.  The symmetric mixed product (FP32 pair terms in
paired lanes, rpy_sym_mixed_x2) against the oracle at the mixed bar 1e-5,
with the FP64 and double-float products on the same layout, and a batched
mixed solve on it; the symmetric mixed product with one target per lane
(rpy_sym_mixed) on tiles of 32 and 64 blobs, against the oracle at 1e-5 and
against the paired-lane kernel, and a batched mixed solve on it."""
import numpy as np
import pytest

from paper_2107_10800_gb300 import build, binding, workloads as W
from oracle import mobility as om
from oracle.system import System

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.lib()


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def loose(r, a, wall, precision="fp64"):
    n = len(r)
    s = binding.Solver(eta=1.0, a=a, wall=wall, precision=precision)
    s.set_bodies(r, np.tile([1.0, 0, 0, 0], (n, 1)), np.arange(n + 1), np.zeros((n, 3)), np.zeros((n, 6)),
                 np.arange(n))
    return s


@pytest.mark.parametrize("tile", [32, 64, 128])
@pytest.mark.parametrize("n", [1, 2, 33, 64, 65, 128, 129, 256, 300, 1000])
@pytest.mark.parametrize("wall", [0, 1])
def test_symmetric_product_matches_oracle(tile, n, wall):
    r, lam = W.random_blobs(300 + n, n, a=0.1, wall=wall)
    if n >= 4:  # an overlapping pair and a pair at contact
        r[1] = r[0] + [0.05, 0.1, 0.0]
        r[3] = r[2] + [0.2, 0.0, 0.0]
    s = loose(r, 0.1, wall)
    s.set_mobility_layout(3, tile)
    assert s.mobility_layout()[3] == tile
    u = s.apply_mobility(lam)
    ref = om.mobility_matvec(r, lam, 0.1, 1.0, wall)
    assert rel(u, ref) <= 1e-12
    s.set_mobility_layout(1, 0)
    assert s.mobility_layout()[3] == 0
    assert rel(s.apply_mobility(lam), u) <= 1e-13


def test_symmetric_layout_rejected_where_it_does_not_apply():
    r, _ = W.random_blobs(1, 10, a=0.1)
    for prec in ("mixed", "fp64"):
        s = loose(r, 0.1, 0, prec)
        for tile in (48, 256, 16):
            with pytest.raises(binding.AmError):
                s.set_mobility_layout(3, tile)


@pytest.mark.parametrize("n", [1, 2, 128, 129, 256, 300, 1000])
@pytest.mark.parametrize("wall", [0, 1])
def test_symmetric_mixed_product_matches_oracle(n, wall):
    # FP32 pair terms in paired lanes, both directions per evaluation; the
    # mixed bar 1e-5, and far from the origin so that the hi/lo positions
    # of near pairs matter
    r, lam = W.random_blobs(500 + n, n, a=0.1, wall=wall)
    if n >= 4:
        r[1] = r[0] + [0.05, 0.1, 0.0]
        r[3] = r[2] + [0.2, 0.0, 0.0]
    r = r + np.array([250.0, -125.0, 0.0])
    s = loose(r, 0.1, wall, "mixed")
    s.set_mobility_layout(3, 128)
    assert s.mobility_layout()[3] == 128
    u = s.apply_mobility(lam)
    ref = om.mobility_matvec(r, lam, 0.1, 1.0, wall)
    assert rel(u, ref) <= 1e-5
    # FP64 and double-float products on the same (symmetric) layout
    assert rel(s.apply_mobility_ex(lam, "fp64"), ref) <= 1e-12
    assert rel(s.apply_mobility_ex(lam, "df64"), ref) <= 1e-11


@pytest.mark.parametrize("tile", [32, 64])
@pytest.mark.parametrize("n", [1, 2, 33, 64, 65, 129, 300, 1000])
@pytest.mark.parametrize("wall", [0, 1])
def test_symmetric_mixed_small_tiles_match_oracle(tile, n, wall):
    # one target per lane (rpy_sym_mixed) on tiles of 32 and 64 blobs, far
    # from the origin so that the hi/lo positions of near pairs matter
    r, lam = W.random_blobs(700 + n, n, a=0.1, wall=wall)
    if n >= 4:
        r[1] = r[0] + [0.05, 0.1, 0.0]
        r[3] = r[2] + [0.2, 0.0, 0.0]
    r = r + np.array([250.0, -125.0, 0.0])
    s = loose(r, 0.1, wall, "mixed")
    s.set_mobility_layout(3, tile)
    lay = s.mobility_layout()
    assert lay[3] == tile and lay[0] == 1
    u = s.apply_mobility(lam)
    ref = om.mobility_matvec(r, lam, 0.1, 1.0, wall)
    assert rel(u, ref) <= 1e-5
    # the FP64 and double-float products on the same partial-sum slots
    assert rel(s.apply_mobility_ex(lam, "fp64"), ref) <= 1e-12
    assert rel(s.apply_mobility_ex(lam, "df64"), ref) <= 1e-11


def test_symmetric_mixed_small_tiles_agree_with_paired_lanes():
    # the two symmetric mixed kernels against each other at 3,000 wall blobs
    r, lam = W.random_blobs(17, 3000, a=0.1, wall=1)
    s = loose(r, 0.1, 1, "mixed")
    s.set_mobility_layout(3, 128)
    u128 = s.apply_mobility(lam)
    for tile in (32, 64):
        s.set_mobility_layout(3, tile)
        assert rel(s.apply_mobility(lam), u128) <= 2e-6


def test_batched_mixed_solve_on_small_symmetric_tiles():
    # systems that stop at different iterations write zero partial sums
    ws = [W.chains_free_space(900 + k, n_chains=1 + k % 3, bodies_per_chain=3) for k in range(12)]
    s = binding.Solver.from_workloads(ws, tol=1e-8, precision="mixed", max_iter=2000)
    s.set_mobility_layout(3, 32)
    U, phi, lam, st = s.solve()
    assert s.mobility_layout()[3] == 32
    assert st["status"] == 0 and st["rel_residual"] <= 1e-8
    for k, (w, (Us, ps, ls)) in enumerate(zip(ws, s.split(U, phi, lam))):
        if k % 3:
            continue
        S = System(w)
        lo, uo, po = S.split(S.solve_dense())
        assert rel(Us.ravel(), uo) <= 1e-5, k


def test_batched_mixed_solve_on_symmetric_layout():
    ws = [W.chains_free_space(600 + k, n_chains=1 + k % 3, bodies_per_chain=4) for k in range(20)]
    s = binding.Solver.from_workloads(ws, tol=1e-8, precision="mixed", max_iter=2000)
    s.set_mobility_layout(3, 128)
    U, phi, lam, st = s.solve()
    assert st["status"] == 0 and st["rel_residual"] <= 1e-8
    for k, (w, (Us, ps, ls)) in enumerate(zip(ws, s.split(U, phi, lam))):
        if k % 4:
            continue
        S = System(w)
        lo, uo, po = S.split(S.solve_dense())
        assert rel(Us.ravel(), uo) <= 1e-5, k


def test_batched_solve_on_symmetric_layout():
    ws = [W.chains_free_space(400 + k, n_chains=1, bodies_per_chain=2 + k % 4) for k in range(40)]
    s = binding.Solver.from_workloads(ws, tol=1e-13, precision="fp64", max_iter=2000)
    s.set_mobility_layout(3, 32)
    U, phi, lam, st = s.solve()
    assert s.mobility_layout()[3] == 32
    assert st["status"] == 0 and st["rel_residual"] <= 1e-13
    for k, (w, (Us, ps, ls)) in enumerate(zip(ws, s.split(U, phi, lam))):
        if k % 5:
            continue
        S = System(w)
        lo, uo, po = S.split(S.solve_dense())
        assert rel(Us.ravel(), uo) <= 1e-10, k
        assert rel(ls.ravel(), lo) <= 1e-10, k
