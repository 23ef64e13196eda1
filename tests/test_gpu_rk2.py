"""The explicit midpoint (RK2) step on the GPU (through the C ABI) against
the oracle's midpoint step: passive and active links, the nonlinear
correction at both stages, consecutive steps, several systems in one
handle, and the argument checks."""
import numpy as np
import pytest

from paper_2107_10800_gb300 import build, binding, workloads as W
from oracle import timestep as ots
from oracle.system import System

pytestmark = pytest.mark.gpu

FP64_SOLVE = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.lib()


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_rk2_step_chains_matches_oracle():
    w = W.chains_free_space(1)
    dt = 2e-2
    s = binding.Solver.from_workload(w, tol=1e-13)
    U, phi, lam, st = s.step_rk2(0.0, dt)
    q, th = s.bodies()
    qo, tho, info = ots.midpoint_step(w, w["q"], w["theta"], 0.0, dt, delta=1e-10, solve_tol=1e-13)
    assert st["status"] == 0
    assert rel(q, qo) <= FP64_SOLVE
    assert rel(th, tho) <= FP64_SOLVE
    assert rel(U, info["U"]) <= FP64_SOLVE  # the midpoint velocities
    assert st["g2_after"] < 1e-20


def test_rk2_step_colony_with_correction_matches_oracle():
    # the midpoint reconstruction is accurate: take the first step size at
    # which the final constraint violation reaches delta = 1e-10
    w = W.diatom_colony(5, n_rods=6, nx=8)
    t = 0.1
    for dt in (2e-2, 4e-2, 6e-2, 8e-2):
        qo, tho, info = ots.midpoint_step(w, w["q"], w["theta"], t, dt, delta=1e-10, solve_tol=1e-13)
        if info["g2_before"] >= 1e-10:
            break
    assert info["g2_before"] >= 1e-10  # the final correction ran
    s = binding.Solver.from_workload(w, t=t, tol=1e-13)
    half = w["dl"](t + 0.5 * dt)
    nxt = w["dl"](t + dt)[:2]
    U, phi, lam, st = s.step_rk2(t, dt, dl_half=half, dl_next=nxt)
    q, th = s.bodies()
    assert st["g2_before"] == pytest.approx(info["g2_before"], rel=1e-6)
    assert st["corr_iterations"] >= 1 and st["g2_after"] < 1e-20
    assert rel(q, qo) <= FP64_SOLVE
    assert rel(th, tho) <= FP64_SOLVE
    assert rel(U, info["U"]) <= FP64_SOLVE


def test_two_rk2_steps_colony_match_oracle():
    w = W.diatom_colony(7, n_rods=4, nx=8)
    t0, dt = 0.05, 1e-2
    s = binding.Solver.from_workload(w, t=t0, tol=1e-13)
    qo, tho = w["q"], w["theta"]
    for k in range(2):
        t = t0 + k * dt
        if k:
            dlp, dlq, dlpd, dlqd = w["dl"](t)
            s.set_constraints(w["body_p"], w["body_q"], dlp, dlq, dlpd, dlqd)
        s.step_rk2(t, dt, dl_half=w["dl"](t + 0.5 * dt), dl_next=w["dl"](t + dt)[:2])
        qo, tho, _ = ots.midpoint_step(w, qo, tho, t, dt, delta=1e-10, solve_tol=1e-13)
    q, th = s.bodies()
    assert rel(q, qo) <= FP64_SOLVE
    assert rel(th, tho) <= FP64_SOLVE


def test_rk2_step_two_systems_match_oracle():
    ws = [W.chains_free_space(2, n_chains=2), W.chains_free_space(3, n_chains=1, bodies_per_chain=5)]
    dt = 2e-2
    s = binding.Solver.from_workloads(ws, tol=1e-13)
    s.step_rk2(0.0, dt)
    for k, w in enumerate(ws):
        q, th = s.bodies(k)
        qo, tho, _ = ots.midpoint_step(w, w["q"], w["theta"], 0.0, dt, delta=1e-10, solve_tol=1e-13)
        assert rel(q, qo) <= FP64_SOLVE
        assert rel(th, tho) <= FP64_SOLVE


def test_rk2_mixed_precision_step():
    # mixed pair arithmetic: the step matches the FP64 oracle to the mixed bar
    w = W.diatom_colony(8, n_rods=4, nx=8)
    t, dt = 0.02, 1e-2
    s = binding.Solver.from_workload(w, t=t, tol=1e-10, precision="mixed")
    s.step_rk2(t, dt, dl_half=w["dl"](t + 0.5 * dt), dl_next=w["dl"](t + dt)[:2])
    q, th = s.bodies()
    qo, tho, _ = ots.midpoint_step(w, w["q"], w["theta"], t, dt, delta=1e-10, solve_tol=1e-12)
    assert rel(q, qo) <= 1e-5
    assert rel(th, tho) <= 1e-5


def test_rk2_argument_checks():
    w = W.diatom_colony(9, n_rods=2, nx=4)
    t, dt = 0.0, 1e-2
    s = binding.Solver.from_workload(w, t=t)
    with pytest.raises(binding.AmError) as e:
        s.step_rk2(t, dt, dl_half=w["dl"](t + 0.5 * dt)[:2])  # active links without derivatives
    assert e.value.code == binding.AM_ERR_ARG
    with pytest.raises(binding.AmError) as e:
        s.step_rk2(t, -dt)
    assert e.value.code == binding.AM_ERR_ARG
    c = W.chains_free_space(1)
    sc = binding.Solver.from_workload(c)
    S = System(c)
    z = np.zeros_like(S.dl_p)
    with pytest.raises(binding.AmError) as e:
        sc.step_rk2(0.0, dt, dl_half=(S.dl_p, S.dl_q, z, z))  # passive links with derivatives
    assert e.value.code == binding.AM_ERR_ARG
