"""Initial guess of the time-step solves from the solution history
(am_set_initial_guess) on the GPU: whatever the order, the trajectory is the
oracle's within the FP64 bar (Euler steps of linked chains, midpoint steps
of a colony with time-dependent sliding links); the extrapolations through the last two or
three solutions take fewer GMRES iterations than the previous solution;
orders outside 0..3 are errors."""
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


def euler_run(w, order, steps, dt, tol, precision="fp64"):
    s = binding.Solver.from_workload(w, t=0.0, tol=tol, precision=precision, max_iter=2000)
    s.set_initial_guess(order)
    its, r0 = [], []
    for k in range(steps):
        t = k * dt
        if k:
            dlp, dlq, dlpd, dlqd = w["dl"](t)
            s.set_constraints(w["body_p"], w["body_q"], dlp, dlq, dlpd, dlqd)
        U, phi, lam, st = s.step(t, dt, dl_next=w["dl"](t + dt)[:2])
        assert st["status"] == 0
        its.append(st["iterations"])
        r0.append(st["rel_residual0"])
    q, th = s.bodies()
    return q, th, its, r0


def test_extrapolated_guess_keeps_the_oracle_trajectory():
    # passive ball joints (B = 0): every step's system is consistent
    w = W.chains_free_space(1)
    dt, steps = 1e-2, 4
    S0 = System(w)
    dl0 = (S0.dl_p, S0.dl_q, None, None)
    qo, tho = w["q"], w["theta"]
    for k in range(steps):
        qo, tho, _ = ots.euler_step(w, qo, tho, k * dt, dt, delta=1e-10, solve_tol=1e-13, dl_now=dl0)
    for order in (0, 1, 2, 3):
        s = binding.Solver.from_workload(w, tol=1e-12, max_iter=2000)
        s.set_initial_guess(order)
        for k in range(steps):
            U, phi, lam, st = s.step(k * dt, dt)
            assert st["status"] == 0, (order, k)
        q, th = s.bodies()
        assert rel(q, qo) <= FP64_SOLVE, order
        assert rel(th, tho) <= FP64_SOLVE, order


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_extrapolation_starts_closer_and_iterates_less(precision):
    # smooth motion over small steps: lambda and U of the previous solution
    # are O(dt) off, of the linear extrapolation O(dt^2), of the quadratic
    # one O(dt^3) (phi, taken from the previous solution, is cheap for the
    # preconditioner to correct)
    w = W.diatom_colony(3, n_rods=8, nx=20)
    dt, steps = 1e-3, 6
    runs = {order: euler_run(w, order, steps, dt, tol=1e-8, precision=precision) for order in (1, 2, 3)}
    its = {o: sum(runs[o][2][3:]) for o in (1, 2, 3)}
    if precision == "fp64":
        assert its[3] < its[2] < its[1], its
    else:  # the refinement's outer steps need not drop with every guess
        assert its[3] <= its[1], its


def test_extrapolated_midpoint_steps_match_oracle():
    # stages at t and t + dt/2 enter the history with their own times.  The
    # stage systems of this colony are consistent only to about 1e-10 after
    # the first stage (prescribed sliding against the reconstructed pose;
    # the oracle's dense solve leaves 5e-11), and restarted GMRES stalls
    # above that (measured on GB300 after 400 iterations: 4.4e-10 in the
    # first step, 2.3e-9 in the second), so a stage may stop at the step
    # budget; the poses still agree.  The stage residuals reached with the
    # extrapolated guess are checked against those of the same steps from
    # the previous solution (order 1): a guess that left the stage solves
    # far above the plain guess's level is caught.
    w = W.diatom_colony(7, n_rods=4, nx=8)
    t0, dt = 0.05, 1e-2
    resid, poses = {}, {}
    for order in (1, 3):
        s = binding.Solver.from_workload(w, t=t0, tol=1e-12, max_iter=400)
        s.set_initial_guess(order)
        resid[order] = []
        for k in range(2):
            t = t0 + k * dt
            if k:
                dlp, dlq, dlpd, dlqd = w["dl"](t)
                s.set_constraints(w["body_p"], w["body_q"], dlp, dlq, dlpd, dlqd)
            U, phi, lam, st = s.step_rk2(t, dt, dl_half=w["dl"](t + 0.5 * dt), dl_next=w["dl"](t + dt)[:2])
            assert st["status"] in (0, binding.AM_ERR_NOT_CONVERGED)
            resid[order].append(st["rel_residual"])  # the larger of the two stages
        poses[order] = s.bodies()
        s.close()
    for r3, r1 in zip(resid[3], resid[1]):
        assert r3 <= max(10 * r1, 1e-12), (resid[3], resid[1])
    qo, tho = w["q"], w["theta"]
    for k in range(2):
        qo, tho, _ = ots.midpoint_step(w, qo, tho, t0 + k * dt, dt, delta=1e-10, solve_tol=1e-13)
    for order in (1, 3):
        q, th = poses[order]
        assert rel(q, qo) <= FP64_SOLVE
        assert rel(th, tho) <= FP64_SOLVE


def test_repeated_time_falls_back_to_the_previous_solution():
    # every step given t = 0: the history times coincide, so the guess is the
    # previous solution and the steps are those of order 1.  The product's
    # layout is fixed (the autotuner's pick, and with it the rounding of the
    # sums, may differ between handles), so the runs are the same
    # computation: a second order-1 run repeats the first exactly.
    w = W.diatom_colony(5, n_rods=4, nx=8)
    dt = 1e-2
    out = {}
    for key, order in (("1", 1), ("1 again", 1), ("3", 3)):
        s = binding.Solver.from_workload(w, t=0.0, tol=1e-12, max_iter=2000)
        s.set_mobility_layout(1, 0)
        s.set_initial_guess(order)
        r0 = []
        for k in range(4):
            U, phi, lam, st = s.step(0.0, dt)
            r0.append(st["rel_residual0"])
        out[key] = (s.bodies(), r0)
    (q1, th1), r01 = out["1"]
    (q3, th3), r03 = out["3"]
    assert out["1 again"][1] == r01
    assert rel(q3, q1) <= FP64_SOLVE and rel(th3, th1) <= FP64_SOLVE
    assert np.allclose(r03, r01, rtol=1e-6, atol=0.0)


def test_initial_guess_order_checks():
    s = binding.Solver.from_workload(W.chains_free_space(1))
    for bad in (-1, 4):
        with pytest.raises(binding.AmError) as e:
            s.set_initial_guess(bad)
        assert e.value.code == binding.AM_ERR_ARG
