"""Pins of the oracle of the learned warm start: the analytic MLP gradient
against finite differences, and the invariances the body-frame features are
built to have."""
import numpy as np

from oracle import mlp
from oracle.kinematics import quat_mul, quat_from_rotvec, rotation_matrix
from paper_2107_10800_gb300 import workloads as W


def small_params(seed=0, scale=0.1):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(mlp.n_params()) * scale


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((5, mlp.FEAT))
    T = rng.standard_normal((5, mlp.OUT))
    mu = rng.standard_normal(mlp.FEAT) * 0.1
    sd = 1.0 + rng.random(mlp.FEAT)
    so = 0.5 + rng.random(mlp.OUT)
    p = small_params()
    loss, g = mlp.loss_and_grad(p, X, T, mu, sd, so)
    idx = rng.choice(len(p), 60, replace=False)
    for k in idx:
        e = np.zeros_like(p); e[k] = 1e-6
        fd = (mlp.loss_and_grad(p + e, X, T, mu, sd, so)[0] - mlp.loss_and_grad(p - e, X, T, mu, sd, so)[0]) / 2e-6
        assert abs(fd - g[k]) <= 1e-7 + 1e-5 * abs(g[k])


def test_features_rigid_motion_invariant():
    w = W.chains_free_space(2)
    M = len(w["q"])
    Nb = w["blob_offset"][-1]
    rng = np.random.default_rng(2)
    U = rng.standard_normal((M, 6))
    lam = rng.standard_normal((Nb, 3))
    sysb = np.zeros(M, int)
    X0 = mlp.features(w["q"], w["theta"], w["F"], w["blob_offset"], U, sysb, 0, lam, w["assembly"],
                      0.1, 1.0)
    assert np.abs(X0[:, 126:138]).max() > 0  # four chains: far flow present
    # rotate and translate everything rigidly (forces, velocities with it)
    rot = quat_from_rotvec(np.array([0.3, -0.7, 0.2]))
    Rr = rotation_matrix(rot)
    q2 = w["q"] @ Rr.T + np.array([5.0, -2.0, 1.0])
    th2 = quat_mul(np.broadcast_to(rot, w["theta"].shape), w["theta"])
    F2 = np.concatenate([w["F"][:, :3] @ Rr.T, w["F"][:, 3:] @ Rr.T], axis=1)
    U2 = np.concatenate([U[:, :3] @ Rr.T, U[:, 3:] @ Rr.T], axis=1)
    X2 = mlp.features(q2, th2, F2, w["blob_offset"], U2, sysb, 0, lam @ Rr.T, w["assembly"], 0.1, 1.0)
    assert np.abs(X0 - X2).max() < 1e-12


def test_far_flow_is_the_oseen_flow_of_other_assemblies():
    # one body far from a forced body of another articulated body: u_far is
    # the Oseen flow of the force and J its gradient (to O(a^2/r^2) and the
    # O(h^2/r^2) of the central difference); bodies of the same articulated
    # body do not count
    q = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [12.0, -4.0, 6.0]])
    f = np.array([[0.0, 0.0, 0.0], [3.0, 1.0, -2.0], [1.0, -2.0, 0.5]])
    th = np.tile([1.0, 0.0, 0.0, 0.0], (3, 1))  # body frames = lab frame
    u, J = mlp.far_flow(q, th, f, np.zeros(3, int), np.array([0, 0, 1]), 0.1, 1.0, 0)

    def oseen(d, g):
        r = np.linalg.norm(d)
        return (g + d * (d @ g) / r ** 2) / (8 * np.pi * r)

    d = q[0] - q[2]
    # RPY differs from Oseen by O(a^2 / r^2) ~ 5e-5 at r = 14
    assert np.allclose(u[0], oseen(d, f[2]), rtol=2e-4)
    # analytic gradient of the Oseen flow by a fine difference of the formula
    Jo = np.stack([(oseen(d + 1e-6 * e, f[2]) - oseen(d - 1e-6 * e, f[2])) / 2e-6 for e in np.eye(3)], axis=1)
    assert np.abs(J[0] - Jo).max() < 1e-2 * np.abs(Jo).max()
    # body 2 feels bodies 0 and 1, body 1 only body 2
    assert np.allclose(u[1], oseen(q[1] - q[2], f[2]), rtol=2e-4)
    assert np.allclose(u[2], oseen(q[2] - q[0], f[0]) + oseen(q[2] - q[1], f[1]), rtol=2e-4)


def test_far_flow_cutoff():
    # sources beyond FAR_R of the body do not count, those inside do
    th = np.tile([1.0, 0.0, 0.0, 0.0], (3, 1))
    f = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 3.0], [1.0, 2.0, 3.0]])
    q = np.array([[0.0, 0.0, 0.0], [mlp.FAR_R - 0.5, 0.0, 0.0], [0.0, mlp.FAR_R + 0.5, 0.0]])
    u, J = mlp.far_flow(q, th, f, np.zeros(3, int), np.arange(3), 0.1, 1.0, 0)
    d = q[0] - q[1]
    r = np.linalg.norm(d)
    expect = (f[1] + d * (d @ f[1]) / r ** 2) / (8 * np.pi * r)
    assert np.allclose(u[0], expect, rtol=1e-4)


def test_features_layout():
    w = W.chains_free_space(3, n_chains=1, bodies_per_chain=3)
    M = len(w["q"])
    X = mlp.features(w["q"], np.tile([1.0, 0, 0, 0], (M, 1)), w["F"], w["blob_offset"],
                     np.zeros((M, 6)), np.zeros(M, int), 0, np.ones((36, 3)), w["assembly"], 0.1, 1.0)
    # identity orientations: relative quaternions are the identity
    assert np.allclose(X[:, 3:7][:, 0], 1.0) and np.allclose(X[:, 3:7][:, 1:], 0.0)
    # two other bodies, 14 empty slots, then the scalar block; one chain:
    # no far flow; zeros to the end
    assert np.all(X[:, 14:7 * 16] == 0.0)
    assert np.allclose(X[:, 7 * 16 + 13], np.log(12) / 5)
    assert np.all(X[:, 7 * 16 + 14:] == 0.0) and X.shape[1] == 144
    # nearest first
    d1 = np.linalg.norm(X[:, 0:3], axis=1)
    d2 = np.linalg.norm(X[:, 7:10], axis=1)
    assert np.all(d1 <= d2)


def _cloud(n=200, seed=5):
    # well-spread body-frame offsets filling a box (points on one quadric
    # surface make 3 of the quadratic flows dependent on the translations)
    return np.random.default_rng(seed).uniform(-1.0, 1.0, (n, 3)) * np.array([1.0, 0.5, 0.5])


def test_flow_basis_structure():
    # each column is a velocity field on the offsets; its velocity gradient
    # (exact for polynomials of degree <= 2 from central differences) has the
    # structure its name says
    rng = np.random.default_rng(6)
    d0 = rng.standard_normal(3) * 0.3
    h = 1e-3

    def field(d):
        return mlp.flow_basis(d[None, :]).reshape(3, mlp.NFLOW)

    grad = np.stack([(field(d0 + h * e) - field(d0 - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
    # grad[c, j, k] = d u_c / d d_j of column k
    for k in range(3):  # translations: constant e_k
        assert np.allclose(field(d0)[:, k], np.eye(3)[k]) and np.allclose(grad[:, :, k], 0)
    for k in range(3, 6):  # rotations: rigid, u = w x d with w = e_(k-3)
        G = grad[:, :, k]
        assert np.allclose(G, -G.T, atol=1e-9)
        w = np.eye(3)[k - 3]
        assert np.allclose(field(d0)[:, k], np.cross(w, d0))
    strain_grads = []
    for k in range(6, 11):  # strains: symmetric traceless gradient, linear
        G = grad[:, :, k]
        assert np.allclose(G, G.T, atol=1e-9) and abs(np.trace(G)) < 1e-9
        assert np.allclose(field(d0)[:, k], G @ d0, atol=1e-9)
        strain_grads.append(G.ravel())
    assert np.linalg.matrix_rank(np.array(strain_grads)) == 5
    for k in range(11, 29):  # quadratics: one component, zero flow and gradient at 0
        assert np.allclose(field(np.zeros(3))[:, k], 0)
        assert np.count_nonzero(np.abs(field(d0)[:, k]) > 0) == 1
    # all 29 independent on a spread cloud; on an ellipsoid surface
    # sum_i d_i^2 / s_i^2 = 1 ties one quadratic combination per component to
    # the translation
    assert np.linalg.matrix_rank(mlp.flow_basis(_cloud())) == mlp.NFLOW
    shell = W._fibonacci_ellipsoid(200, (1.0, 0.5, 0.5))
    assert np.linalg.matrix_rank(mlp.flow_basis(shell)) == mlp.NFLOW - 3


def test_flow_targets_recover_a_flow_in_the_span():
    rho = _cloud()
    off = np.array([0, len(rho)])
    rng = np.random.default_rng(7)
    c = rng.standard_normal(mlp.NFLOW)
    theta = quat_from_rotvec(np.array([0.4, 0.1, -0.9]))[None, :]
    R = rotation_matrix(theta)[0]
    u_lab = (mlp.flow_basis(rho) @ c).reshape(-1, 3) @ R.T
    T0 = mlp.flow_targets(theta, rho, off, u_lab, ridge=0.0)
    assert np.abs(T0[0, :mlp.NFLOW] - c).max() < 1e-10 and np.all(T0[0, mlp.NFLOW:] == 0)
    T1 = mlp.flow_targets(theta, rho, off, u_lab)
    assert np.abs(T1[0, :mlp.NFLOW] - c).max() < 1e-3 * np.abs(c).max()
    # the flow of the coefficients is the flow that was fitted
    assert np.abs(mlp.flow_field(theta, rho, off, T0) - u_lab).max() < 1e-10


def test_flow_targets_rigid_motion_invariant():
    rho = np.concatenate([_cloud(60), _cloud(40) * 0.5])
    off = np.array([0, 60, 100])
    rng = np.random.default_rng(8)
    theta = np.stack([quat_from_rotvec(rng.standard_normal(3)) for _ in range(2)])
    u = rng.standard_normal((100, 3))
    T0 = mlp.flow_targets(theta, rho, off, u)
    rot = quat_from_rotvec(np.array([-0.3, 0.8, 0.5]))
    Rr = rotation_matrix(rot)
    T1 = mlp.flow_targets(quat_mul(np.broadcast_to(rot, theta.shape), theta), rho, off, u @ Rr.T)
    assert np.abs(T0 - T1).max() < 1e-12


def test_background_flow_far_field_is_a_stokeslet():
    # two bodies 200 apart in free space: the flow of the far body at the
    # near one is the Oseen tensor of its total force, to O(size / distance)
    from oracle.mobility import mobility_dense
    rho = _cloud(30) * 0.5
    r = np.concatenate([rho, rho + np.array([200.0, 30.0, -50.0])])
    off = np.array([0, 30, 60])
    lam = np.random.default_rng(9).standard_normal((60, 3))
    Md = mobility_dense(r, 0.1, 1.0, 0)
    u = mlp.background_flow(Md, lam, off).reshape(-1, 3)
    d = np.array([-200.0, -30.0, 50.0])
    rn = np.linalg.norm(d)
    O = (np.eye(3) + np.outer(d, d) / rn ** 2) / (8 * np.pi * rn)
    expect = O @ lam[30:].sum(axis=0)
    assert np.abs(u[:30] - expect).max() < 0.02 * np.abs(expect).max()
    # a body alone feels no background flow
    u1 = mlp.background_flow(Md[:90, :90], lam[:30], off[:2])
    assert np.all(u1 == 0)


def test_exact_background_flow_makes_the_block_diagonal_solve_exact():
    # x0 = P~^-1 (u_s - u_ext, -F, B) with the exact u_ext = (M - M~) lambda
    # of the solution is the solution itself (every body's own equations are
    # exact given the others' flow)
    from oracle.system import System
    w = W.chains_free_space(3, n_chains=2, bodies_per_chain=3)
    S = System(w)
    y = S.solve_dense()
    lam = S.split(y)[0]
    u_ext = mlp.background_flow(S.mobility(), lam, S.off)
    b = S.rhs()
    bt = b.copy()
    bt[:3 * S.Nb] -= u_ext
    x0 = S.apply_preconditioner(bt)
    assert np.abs(x0 - y).max() < 1e-9 * np.abs(y).max()
