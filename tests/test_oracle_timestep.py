"""Pins of the oracle's time step (Sec. 4): reconstruction properties, the
robot-arm model, the O(dt^2) one-step constraint error of explicit Euler, the
correction's convergence and the exactness of its Jacobian (App. B)."""
import numpy as np
import pytest

from oracle import timestep as ts
from oracle.kinematics import rotation_matrix, quat_mul, quat_from_rotvec
from oracle.system import System
from paper_2107_10800_gb300 import workloads


def test_rotation_matrix_properties():
    rng = np.random.default_rng(0)
    th = rng.standard_normal((10, 4))
    th /= np.linalg.norm(th, axis=1, keepdims=True)
    R = rotation_matrix(th)
    for Rk in R:
        assert np.allclose(Rk @ Rk.T, np.eye(3), atol=1e-15)
        assert abs(np.linalg.det(Rk) - 1) < 1e-14
    # composition (Eq. quaternion_mult): R(t2 . t1) = R(t2) R(t1)
    R12 = rotation_matrix(quat_mul(th[:5], th[5:]))
    assert np.allclose(R12, R[:5] @ R[5:], atol=1e-14)


def test_rotation_vector_quaternion_is_rodrigues():
    # theta_gamma rotates by |gamma| about gamma (textbook Rodrigues formula).
    rng = np.random.default_rng(1)
    for _ in range(5):
        g = rng.standard_normal(3)
        ang = np.linalg.norm(g)
        k = g / ang
        Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        Rr = np.eye(3) + np.sin(ang) * Kx + (1 - np.cos(ang)) * Kx @ Kx
        assert np.allclose(rotation_matrix(quat_from_rotvec(g)), Rr, atol=1e-14)


def open_chain():
    return workloads.chains_free_space(3, n_chains=1, bodies_per_chain=6)


def test_reconstruction_rank_and_zero_com():
    # rank P^a = 3 (M_a - 1), and -(P^a)^+ z^a has zero centre (Sec. 4.1).
    w = open_chain()
    S = System(w)
    for a_, (bodies, links) in ts.assemblies_of(S.assembly, S.bp).items():
        Ps = ts.connectivity_scalar(bodies, links, S.bp, S.bq)
        assert 3 * np.linalg.matrix_rank(Ps) == 3 * (len(bodies) - 1)
    q_com = {0: np.array([1.0, 2.0, 3.0])}
    q = ts.reconstruct(q_com, S.theta, S.dl_p, S.dl_q, S.assembly, S.bp, S.bq)
    assert np.allclose(q.mean(axis=0), q_com[0], atol=1e-14)


def test_reconstruction_equals_robot_arm():
    # Open chains: the pseudo-inverse reconstruction is the robot-arm model
    # (Eq. robot-arm) with the same centre (Sec. 4.1).
    w = open_chain()
    S = System(w)
    rng = np.random.default_rng(2)
    th = quat_mul(quat_from_rotvec(0.3 * rng.standard_normal((S.M_bodies, 3))), S.theta)
    R = rotation_matrix(th)
    arm = [np.zeros(3)]
    for k in range(S.P):  # link k joins body k (p) and k+1 (q)
        arm.append(arm[-1] + R[k] @ S.dl_p[k] - R[k + 1] @ S.dl_q[k])
    arm = np.array(arm)
    c = np.array([0.5, -1.0, 2.0])
    arm += c - arm.mean(axis=0)
    q = ts.reconstruct({0: c}, th, S.dl_p, S.dl_q, S.assembly, S.bp, S.bq)
    assert np.abs(q - arm).max() <= 1e-13
    assert np.abs(ts.constraint_g(q, th, S.dl_p, S.dl_q, S.bp, S.bq)).max() <= 1e-13


def test_correction_jacobian_matches_finite_differences():
    w = workloads.diatom_colony(1, n_rods=4, nx=6)
    S = System(w, t=0.1)
    bodies, links = ts.assemblies_of(S.assembly, S.bp)[0]
    col = {int(b): k for k, b in enumerate(bodies)}
    R = rotation_matrix(S.theta)
    lt_p = np.einsum("nab,nb->na", R[S.bp], S.dl_p)
    lt_q = np.einsum("nab,nb->na", R[S.bq], S.dl_q)
    qpair = np.stack([S.q[S.bp], S.q[S.bq]], axis=1)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(7 * len(bodies)) * 0.3
    J = ts.correction_jacobian(x, lt_p, lt_q, S.bp, S.bq, col)
    eps = 1e-6
    for k in range(len(x)):
        e = np.zeros_like(x); e[k] = eps
        fd = (ts.correction_residual(x + e, qpair, lt_p, lt_q, S.bp, S.bq, col)
              - ts.correction_residual(x - e, qpair, lt_p, lt_q, S.bp, S.bq, col)) / (2 * eps)
        assert np.abs(fd - J[:, k]).max() <= 1e-7
    # 30 nonzeros per link (App. B) at generic increments: 15 per body side,
    # of which the 12 rotational ones vanish when that side's link vector is
    # zero (the second colony link has dl_q = 0).
    nz = np.count_nonzero(np.abs(J[:3 * len(links)]) > 0)
    expect = sum(30 - 12 * (not np.any(lt_q[k])) - 12 * (not np.any(lt_p[k]))
                 for k in range(len(links)))
    assert nz == expect and expect >= 18 * len(links)


def colony_state(seed=1, n_rods=6, nx=10):
    w = workloads.diatom_colony(seed, n_rods=n_rods, nx=nx)
    return w


@pytest.mark.slow
def test_euler_constraint_error_is_second_order():
    # Sec. 4.2: without correction the one-step constraint error of explicit
    # Euler decays as dt^2.
    w = colony_state()
    errs = []
    for dt in (4e-3, 2e-3, 1e-3):
        _, _, info = ts.euler_step(w, w["q"], w["theta"], 0.2, dt, delta=np.inf)
        errs.append(np.sqrt(info["g2_before"]))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8) and np.all(rates < 2.2), (errs, rates)


@pytest.mark.slow
def test_correction_converges_fast():
    # Sec. 4.2 / 4.3: the correction brings ||g||^2 below delta in fewer than
    # five iterations.
    w = colony_state()
    q, th, info = ts.euler_step(w, w["q"], w["theta"], 0.2, 5e-2, delta=1e-10)
    assert info["g2_before"] >= 1e-10
    assert info["g2_after"] < 1e-20
    assert max(info["corr_iters"].values()) < 5
    # unit quaternions preserved to the tolerance
    assert np.abs(np.linalg.norm(th, axis=1) - 1).max() < 1e-10


def test_open_chain_needs_no_correction():
    w = open_chain()
    q, th, info = ts.euler_step(w, w["q"], w["theta"], 0.0, 1e-2, delta=1e-10)
    assert info["g2_before"] < 1e-24
    assert info["corr_iters"] == {}


def _two_free_bodies():
    # two icosahedral shells 2.6 apart in free space under constant forces
    # and torques: the motion is nonlinear only through their hydrodynamic
    # coupling, which is smooth at this separation
    from oracle.kinematics import quat_from_rotvec
    ico = workloads.icosahedron(0.5)
    q = np.array([[0.0, 0.0, 0.0], [2.5, 0.5, -0.3]])
    th = np.stack([quat_from_rotvec(np.array([0.3, 0.2, -0.1])), quat_from_rotvec(np.array([-0.5, 0.1, 0.7]))])
    F = np.array([[1.0, 0.5, -0.2, 0.3, -0.4, 0.8], [-0.7, 0.2, 0.4, -0.6, 0.5, 0.2]])
    return dict(name="two", eta=1.0, a=0.1, wall=0, q=q, theta=th, blob_offset=np.array([0, 12, 24]),
                rho=np.concatenate([ico, ico]), F=F, assembly=np.array([0, 1]),
                body_p=np.zeros(0, int), body_q=np.zeros(0, int), joints=np.zeros((0, 3)), dl=None)


def _integrate(stepper, w, T, N):
    # passive links: body-frame link vectors from the joints at the initial
    # pose, kept for every step
    S0 = System(w)
    dl0 = (S0.dl_p, S0.dl_q, None, None)
    q, th = w["q"].copy(), w["theta"].copy()
    dt = T / N
    for k in range(N):
        q, th, _ = stepper(w, q, th, k * dt, dt, solve_tol=1e-13, dl_now=dl0)
    return q, th


def test_midpoint_step_is_second_order_and_euler_first():
    # error at T against a 128-step midpoint reference, halving dt: the
    # explicit midpoint scheme (App. "Midpoint scheme") divides the error by
    # 4, Euler (Sec. 4.3) by 2
    w = _two_free_bodies()
    T = 2.0
    qr, thr = _integrate(ts.midpoint_step, w, T, 128)
    for stepper, lo, hi in ((ts.midpoint_step, 3.6, 4.5), (ts.euler_step, 1.85, 2.15)):
        errs = []
        for N in (4, 8, 16):
            q, th = _integrate(stepper, w, T, N)
            errs.append(max(np.abs(q - qr).max(), np.abs(th - thr).max()))
        for e1, e2 in zip(errs, errs[1:]):
            assert lo < e1 / e2 < hi, (stepper.__name__, errs)


def test_midpoint_step_beats_euler_on_a_chain():
    # three linked shells: the same number of steps is more accurate with
    # the midpoint scheme, and the links stay closed (ball joints)
    w = workloads.chains_free_space(3, n_chains=1, bodies_per_chain=3)
    T = 2.0
    qr, _ = _integrate(ts.midpoint_step, w, T, 64)
    qm, thm = _integrate(ts.midpoint_step, w, T, 8)
    qe, _ = _integrate(ts.euler_step, w, T, 8)
    assert np.abs(qm - qr).max() < 0.5 * np.abs(qe - qr).max()
    S = System(w)
    g = ts.constraint_g(qm, thm, S.dl_p, S.dl_q, S.bp, S.bq)
    assert np.abs(g).max() < 1e-9
