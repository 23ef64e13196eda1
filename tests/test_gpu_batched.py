"""The batched form: several independent suspensions of different sizes in
one handle, solved together (per-system GMRES in lockstep, block-diagonal
mobility product).  Every system must match the oracle's solution of that
system alone."""
import numpy as np
import pytest

from paper_2107_10800_gb300 import build, binding, workloads as W
from oracle.system import System
from oracle import timestep as ots

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.lib()


def rel(a, b):
    a = np.asarray(a, float).ravel()
    b = np.asarray(b, float).ravel()
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def chain_batch():
    return [W.chains_free_space(11, n_chains=1, bodies_per_chain=3),
            W.chains_free_space(12, n_chains=3, bodies_per_chain=5),
            W.chains_free_space(13, n_chains=2, bodies_per_chain=8)]


def test_batched_solve_matches_each_system():
    ws = chain_batch()
    s = binding.Solver.from_workloads(ws, tol=1e-13)
    U, phi, lam, st = s.solve()
    assert st["status"] == 0 and st["rel_residual"] <= 1e-13
    for w, (Us, ps, ls) in zip(ws, s.split(U, phi, lam)):
        S = System(w)
        lo, uo, po = S.split(S.solve_dense())
        assert rel(Us, uo) <= 1e-10
        assert rel(ls, lo) <= 1e-10
        assert rel(ps, po) <= 1e-10


def test_batched_equals_separate_solves():
    ws = chain_batch()
    s = binding.Solver.from_workloads(ws, tol=1e-13)
    U, phi, lam, _ = s.solve()
    for w, (Us, ps, ls) in zip(ws, s.split(U, phi, lam)):
        U1, p1, l1, _ = binding.Solver.from_workload(w, tol=1e-13).solve()
        assert rel(Us, U1) <= 1e-11 and rel(ls, l1) <= 1e-11


def test_batched_mixed_matches_each_system():
    ws = chain_batch()
    s = binding.Solver.from_workloads(ws, tol=1e-8, precision="mixed")
    U, phi, lam, st = s.solve()
    assert st["status"] == 0 and st["rel_residual"] <= 1e-8
    for w, (Us, ps, ls) in zip(ws, s.split(U, phi, lam)):
        S = System(w)
        lo, uo, po = S.split(S.solve_dense())
        assert rel(Us, uo) <= 1e-5
        assert rel(ls, lo) <= 1e-5


def test_batched_colonies_step_with_active_links():
    ws = [W.diatom_colony(21, n_rods=4, nx=6), W.diatom_colony(22, n_rods=6, nx=8)]
    t, dt = 0.1, 2e-2
    s = binding.Solver.from_workloads(ws, t=t, tol=1e-13)
    nxt = [w["dl"](t + dt)[:2] for w in ws]
    dlp1 = np.concatenate([a for a, _ in nxt])
    dlq1 = np.concatenate([b for _, b in nxt])
    U, phi, lam, st = s.step(t, dt, dl_next=(dlp1, dlq1))
    assert st["status"] == 0 and st["corr_iterations"] >= 1
    for k, w in enumerate(ws):
        q, th = s.bodies(system=k)
        qo, tho, info = ots.euler_step(w, w["q"], w["theta"], t, dt, delta=1e-10, solve_tol=1e-13)
        assert rel(q, qo) <= 1e-10
        assert rel(th, tho) <= 1e-10


def test_batched_workload_solves():
    # a slice of the 256-suspension batch (log-uniform sizes), mixed precision
    ws = W.batched_chains(1, n_systems=8, lo=500, hi=3000)
    s = binding.Solver.from_workloads(ws, tol=1e-8, precision="mixed")
    U, phi, lam, st = s.solve()
    assert st["status"] == 0 and st["rel_residual"] <= 1e-8
    k = int(np.argmin([W.counts(w)[0] for w in ws]))
    S = System(ws[k])
    lo, uo, po = S.split(S.solve_dense())
    Us, ps, ls = s.split(U, phi, lam)[k]
    assert rel(Us, uo) <= 1e-5


def test_partial_batch_is_an_error():
    s = binding.Solver(n_systems=2)
    w = W.chains_free_space(1)
    s.set_bodies(w["q"], w["theta"], w["blob_offset"], w["rho"], w["F"], w["assembly"], system=0)
    with pytest.raises(binding.AmError):
        s.solve()


@pytest.mark.parametrize("precision,tol,bar", [("fp64", 1e-13, 1e-10), ("mixed", 1e-8, 1e-5)])
def test_many_small_systems(precision, tol, bar):
    # 300 systems (more than the 256 threads of the loop-control block, so
    # its per-system loops stride), one short chain each, 2-4 bodies: they
    # stop at different iterations, so the products skip stopped systems and
    # the per-system arrival counts of the Arnoldi kernels and (mixed) the
    # per-system residual bound all see many systems
    ws = [W.chains_free_space(100 + k, n_chains=1, bodies_per_chain=2 + k % 3) for k in range(300)]
    s = binding.Solver.from_workloads(ws, tol=tol, precision=precision, max_iter=2000)
    U, phi, lam, st = s.solve()
    assert st["status"] == 0 and st["rel_residual"] <= tol
    for k, (w, (Us, ps, ls)) in enumerate(zip(ws, s.split(U, phi, lam))):
        if k % 10:  # every tenth system against the oracle's dense solve
            continue
        S = System(w)
        lo, uo, po = S.split(S.solve_dense())
        assert rel(Us, uo) <= bar, k
        assert rel(ls, lo) <= bar, k
