"""Pins of the oracle's blob mobility (Sec. 2.3, Eq. RPY) to facts other
than itself: closed forms, the definition by quadrature, published wall
self-mobilities, limits and matrix properties."""
import numpy as np
import pytest

from oracle.mobility import (rpy_free_pair, rpy_wall_image_pair, pair_tensor,
                             mobility_dense)
from tests.quadrature import oseen, blake, double_average
from paper_2107_10800_gb300 import workloads

A, ETA = 0.1, 1.0
MU0 = 1.0 / (6.0 * np.pi * ETA * A)
DIR = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])


def test_self_mobility_is_stokes_drag():
    # Single blob: the mobility of a sphere of radius a, 1/(6 pi eta a).
    T = rpy_free_pair(np.zeros(3), A, ETA)
    assert np.allclose(T, MU0 * np.eye(3), rtol=1e-15, atol=0)


@pytest.mark.parametrize("r", [0.3, 0.5, 1.7])
def test_free_pair_equals_double_surface_average(r):
    # Eq. RPY by quadrature of the Oseen tensor over both spheres.
    d = r * DIR
    Q = double_average(oseen, np.zeros(3), -d, A, ETA, 16, 32)
    E = rpy_free_pair(d, A, ETA)
    assert np.abs(Q - E).max() <= 1e-12 * np.abs(E).max()


@pytest.mark.parametrize("r", [0.05, 0.15])
def test_overlapping_pair_equals_double_surface_average(r):
    # Overlapping blobs: the integrand is singular on the intersection
    # circle, so the quadrature converges slowly; 1e-3 still separates the
    # overlap formula from any wrong coefficient.
    d = r * DIR
    Q = double_average(oseen, np.zeros(3), -d, A, ETA, 32, 64)
    E = rpy_free_pair(d, A, ETA)
    assert np.abs(Q - E).max() <= 1e-3 * np.abs(E).max()


def test_free_pair_continuous_at_contact():
    lo = rpy_free_pair((2 * A - 1e-12) * DIR, A, ETA)
    hi = rpy_free_pair((2 * A + 1e-12) * DIR, A, ETA)
    rr = np.outer(DIR, DIR)
    expect = MU0 * (7.0 / 16.0 * np.eye(3) + 3.0 / 16.0 * rr)
    assert np.allclose(lo, expect, rtol=1e-10)
    assert np.allclose(hi, expect, rtol=1e-10)


def test_far_field_is_oseen():
    d = 1e4 * DIR
    T = rpy_free_pair(d, A, ETA)
    O = oseen(np.zeros(3), -d, ETA)
    assert np.abs(T - O).max() <= 1e-8 * np.abs(O).max()


@pytest.mark.parametrize("h", [0.12, 0.2, 0.5, 2.0])
def test_wall_self_mobility_closed_form(h):
    # Published self-mobility of a blob above a no-slip wall (Swan & Brady
    # 2007, the wall RPY reference of Sec. 2.3), xi = a/h:
    #   mu_par  = mu0 (1 - 9 xi/16 + xi^3/8 - xi^5/16)
    #   mu_perp = mu0 (1 - 9 xi/8  + xi^3/2 - xi^5/8)
    # whose leading terms are Faxen's and Lorentz's wall corrections.
    x = np.array([0.3, -0.2, h])
    T = pair_tensor(x, x, A, ETA, 1)
    xi = A / h
    par = MU0 * (1 - 9 * xi / 16 + xi ** 3 / 8 - xi ** 5 / 16)
    perp = MU0 * (1 - 9 * xi / 8 + xi ** 3 / 2 - xi ** 5 / 8)
    assert np.allclose(np.diag(T), [par, par, perp], rtol=1e-13)
    off = T - np.diag(np.diag(T))
    assert np.abs(off).max() <= 1e-15 * MU0


def test_blake_tensor_is_blakes():
    # The quadrature reference's Blake tensor: zero on the wall (no slip),
    # divergence-free in x, Oseen-like near the source.
    rng = np.random.default_rng(3)
    for _ in range(5):
        y = np.array([*rng.uniform(-1, 1, 2), rng.uniform(0.2, 2)])
        xw = np.array([[*rng.uniform(-2, 2, 2), 0.0]])
        assert np.abs(blake(xw, y[None], ETA)).max() < 1e-14
        x = np.array([*rng.uniform(-2, 2, 2), rng.uniform(0.2, 2)])
        eps = 1e-5
        div = np.zeros(3)
        for k in range(3):
            e = np.zeros(3); e[k] = eps
            Gp = blake((x + e)[None], y[None], ETA)[0]
            Gm = blake((x - e)[None], y[None], ETA)[0]
            div += (Gp[k, :] - Gm[k, :]) / (2 * eps)
        assert np.abs(div).max() < 1e-6


@pytest.mark.parametrize("case", [
    (np.array([0.0, 0.0, 0.3]), np.array([0.25, 0.1, 0.45])),
    (np.array([0.0, 0.0, 0.15]), np.array([-0.3, 0.2, 0.2])),
    (np.array([0.1, 0.0, 1.0]), np.array([0.2, -0.6, 0.4])),
])
def test_wall_pair_equals_double_surface_average(case):
    # Eq. RPY with Blake's Green's function, by quadrature: checks the
    # symbolic regularisation of the image part.
    xi, xj = case
    Q = double_average(blake, xi, xj, A, ETA, 16, 32)
    E = pair_tensor(xi, xj, A, ETA, 1)
    assert np.abs(Q - E).max() <= 1e-11 * np.abs(E).max()


def test_wall_image_vanishes_far_from_wall():
    # h -> infinity: the wall pair tends to the free-space pair.
    xi = np.array([0.0, 0.0, 1e5])
    xj = np.array([0.3, 0.1, 1e5 + 0.2])
    W = rpy_wall_image_pair(xi, xj, A, ETA)
    F = rpy_free_pair(xi - xj, A, ETA)
    assert np.abs(W).max() <= 1e-4 * np.abs(F).max()


def test_wall_pair_reciprocity():
    # M_ij(x, y) = M_ji(y, x) (the Green's function is reciprocal).
    rng = np.random.default_rng(5)
    x = np.c_[rng.uniform(-1, 1, (20, 2)), rng.uniform(0.15, 1.5, 20)]
    y = np.c_[rng.uniform(-1, 1, (20, 2)), rng.uniform(0.15, 1.5, 20)]
    Mxy = pair_tensor(x, y, A, ETA, 1)
    Myx = pair_tensor(y, x, A, ETA, 1)
    assert np.abs(Mxy - np.swapaxes(Myx, -1, -2)).max() <= 1e-13 * MU0


@pytest.mark.parametrize("wall", [0, 1])
def test_mobility_symmetric_positive_definite(wall):
    # M is symmetric and positive definite, overlaps included (Sec. 2.3).
    r, _ = workloads.random_blobs(7, 300, box=2.0, a=A, wall=wall)
    Mm = mobility_dense(r, A, ETA, wall)
    assert np.abs(Mm - Mm.T).max() <= 1e-15 * np.abs(Mm).max()
    assert np.linalg.eigvalsh(Mm).min() > 0


def test_mobility_pd_config_chains():
    w = workloads.chains_free_space(1)
    from oracle.system import System
    S = System(w)
    Mm = S.mobility()
    assert np.abs(Mm - Mm.T).max() == 0.0
    np.linalg.cholesky(Mm)


def test_wall_rejects_penetrating_blob():
    r = np.array([[0.0, 0.0, 0.5], [1.0, 0.0, 0.1]])
    with pytest.raises(ValueError):
        mobility_dense(r, A, ETA, 1)
