"""Steric repulsion on the GPU (through the C ABI) against the oracle: blob
forces between articulated bodies and with the wall, their effect on a solve
and on a time step, several systems in one handle, and the argument
checks."""
import numpy as np
import pytest

from paper_2107_10800_gb300 import build, binding, learned, workloads as W
from oracle import steric as ost
from oracle import timestep as ots
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


def oracle_forces(w, S, eps, rng, rc, eps_w=0.0, rng_w=1.0):
    return ost.blob_forces(S.r, S.off, w["assembly"], w["a"], eps, rng, rc, w["wall"], eps_w, rng_w)


def with_steric_F(w, S, f):
    """The workload with the steric body forces added to its F."""
    w2 = dict(w)
    w2["F"] = np.asarray(w["F"]) + ost.body_forces(S.r, S.q, S.off, f)
    return w2


def test_forces_free_space_chains_match_oracle():
    w = W.chains_free_space(3)
    S = System(w)
    s = binding.Solver.from_workload(w)
    s.set_repulsion(0.2, 0.1, 3.0)
    fo = oracle_forces(w, S, 0.2, 0.1, 3.0)
    assert np.abs(fo).max() > 0  # chains within the cutoff of each other
    assert rel(s.steric_forces(), fo) <= 1e-12


def test_forces_wall_bacteria_match_oracle():
    w = learned.bacteria_at_density(31, 3)
    S = System(w)
    s = binding.Solver.from_workload(w)
    s.set_repulsion(0.05, 0.1, 9.0, 0.3, 0.2)
    fo = oracle_forces(w, S, 0.05, 0.1, 9.0, 0.3, 0.2)
    assert rel(s.steric_forces(), fo) <= 1e-12
    s.set_repulsion(0.0, 0.0, 0.0)
    assert np.all(s.steric_forces() == 0.0)


def test_solve_with_repulsion_matches_oracle():
    w = W.chains_free_space(4)
    S = System(w)
    f = oracle_forces(w, S, 0.5, 0.2, 4.0)
    So = System(with_steric_F(w, S, f))
    s = binding.Solver.from_workload(w, tol=1e-13)
    s.set_repulsion(0.5, 0.2, 4.0)
    U, phi, lam, st = s.solve()
    _, U_o, _ = So.split(So.solve_dense())
    assert rel(U.ravel(), U_o) <= 1e-10


def test_euler_step_with_repulsion_matches_oracle():
    w = learned.bacteria_at_density(32, 2)
    S = System(w)
    f = oracle_forces(w, S, 0.05, 0.1, 12.0, 0.3, 0.2)
    w2 = with_steric_F(w, S, f)
    dt = 1e-2
    s = binding.Solver.from_workload(w, tol=1e-13)
    s.set_repulsion(0.05, 0.1, 12.0, 0.3, 0.2)
    s.step(0.0, dt)
    q, th = s.bodies()
    dl0 = (S.dl_p, S.dl_q, None, None)
    qo, tho, _ = ots.euler_step(w2, w["q"], w["theta"], 0.0, dt, delta=1e-10, solve_tol=1e-13, dl_now=dl0)
    assert rel(q, qo) <= 1e-10
    assert rel(th, tho) <= 1e-10


def test_forces_two_systems_do_not_interact():
    ws = [W.chains_free_space(5), W.chains_free_space(5)]  # the same suspension twice
    s = binding.Solver.from_workloads(ws)
    s.set_repulsion(0.2, 0.1, 3.0)
    f = s.steric_forces()
    S = System(ws[0])
    fo = oracle_forces(ws[0], S, 0.2, 0.1, 3.0)
    n = len(fo)
    assert rel(f[:n], fo) <= 1e-12 and rel(f[n:], fo) <= 1e-12


def test_repulsion_argument_checks():
    s = binding.Solver.from_workload(W.chains_free_space(6))
    for args in ((-1.0, 0.1, 1.0), (0.1, 0.0, 1.0), (0.1, 0.1, -1.0), (0.1, 0.1, 1.0, 0.2, 0.1)):
        with pytest.raises(binding.AmError) as e:
            s.set_repulsion(*args)  # the last: a wall term without a wall
        assert e.value.code == binding.AM_ERR_ARG
