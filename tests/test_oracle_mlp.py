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
    U = np.random.default_rng(2).standard_normal((M, 6))
    sysb = np.zeros(M, int)
    X0 = mlp.features(w["q"], w["theta"], w["F"], w["blob_offset"], U, sysb, 0)
    # rotate and translate everything rigidly (forces, velocities with it)
    rot = quat_from_rotvec(np.array([0.3, -0.7, 0.2]))
    Rr = rotation_matrix(rot)
    q2 = w["q"] @ Rr.T + np.array([5.0, -2.0, 1.0])
    th2 = quat_mul(np.broadcast_to(rot, w["theta"].shape), w["theta"])
    F2 = np.concatenate([w["F"][:, :3] @ Rr.T, w["F"][:, 3:] @ Rr.T], axis=1)
    U2 = np.concatenate([U[:, :3] @ Rr.T, U[:, 3:] @ Rr.T], axis=1)
    X2 = mlp.features(q2, th2, F2, w["blob_offset"], U2, sysb, 0)
    assert np.abs(X0 - X2).max() < 1e-12


def test_features_layout():
    w = W.chains_free_space(3, n_chains=1, bodies_per_chain=3)
    M = len(w["q"])
    X = mlp.features(w["q"], np.tile([1.0, 0, 0, 0], (M, 1)), w["F"], w["blob_offset"],
                     np.zeros((M, 6)), np.zeros(M, int), 0)
    # identity orientations: relative quaternions are the identity
    assert np.allclose(X[:, 3:7][:, 0], 1.0) and np.allclose(X[:, 3:7][:, 1:], 0.0)
    # two other bodies, 14 empty slots, then the scalar block
    assert np.all(X[:, 14:7 * 16] == 0.0)
    assert np.allclose(X[:, 7 * 16 + 13], np.log(12) / 5)
    assert np.all(X[:, 7 * 16 + 14:] == 0.0)
    # nearest first
    d1 = np.linalg.norm(X[:, 0:3], axis=1)
    d2 = np.linalg.norm(X[:, 7:10], axis=1)
    assert np.all(d1 <= d2)
