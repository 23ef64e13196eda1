"""Pins of the single-blob oracle (generalised RPY tensor, free space): the
rotational far forms against finite-difference vorticity of the pinned
translational tensor and of the rotlet; the overlapping and the separated
forms against quadrature of the surface averages that define the tensor;
continuity at contact and at coincidence, symmetry and positive
definiteness (overlaps included), and the dense against the formal solution
of the constrained problem."""
import numpy as np
import pytest

from oracle import single_blob as sb
from oracle.mobility import rpy_free_pair
from paper_2107_10800_gb300 import workloads as W
from quadrature import rotational_averages

A, ETA = 0.1, 1.3
DIR = np.array([0.36, -0.48, 0.8]) / np.linalg.norm([0.36, -0.48, 0.8])


def curl_half(field, x, h=1e-5):
    """(1/2) curl of the vector field at x by central differences."""
    J = np.zeros((3, 3))  # J[i, k] = d field_i / d x_k
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (field(x + e) - field(x - e)) / (2 * h)
    return 0.5 * np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])


def test_far_rotation_from_force_is_half_the_curl_of_the_rpy_flow():
    rng = np.random.default_rng(0)
    for _ in range(5):
        d = rng.standard_normal(3)
        d *= rng.uniform(2.5 * A, 2.0) / np.linalg.norm(d)
        F = rng.standard_normal(3)
        w = curl_half(lambda x: rpy_free_pair(x, A, ETA) @ F, d)
        assert np.allclose(sb.pair_rt(d, A, ETA) @ F, w, rtol=1e-6, atol=1e-10)


def test_far_rotation_from_torque_is_half_the_curl_of_the_rotlet():
    rng = np.random.default_rng(1)
    for _ in range(5):
        d = rng.standard_normal(3)
        d *= rng.uniform(2.5 * A, 2.0) / np.linalg.norm(d)
        T = rng.standard_normal(3)
        # velocity at x from the torque at the origin: M_tr(x) T
        w = curl_half(lambda x: sb.pair_rt(-x, A, ETA).T @ T, d)
        assert np.allclose(sb.pair_rr(d, A, ETA) @ T, w, rtol=1e-6, atol=1e-10)


def test_continuity_at_contact_and_coincidence():
    e = np.array([0.3, -0.5, 0.8])
    e /= np.linalg.norm(e)
    for f in (sb.pair_rt, sb.pair_rr):
        lo, hi = f(e * (2 * A - 1e-12), A, ETA), f(e * (2 * A + 1e-12), A, ETA)
        assert np.abs(lo - hi).max() < 1e-8 * np.abs(hi).max()
    # r -> 0: the coupling vanishes and rotation tends to the self term
    assert np.abs(sb.pair_rt(e * 1e-12, A, ETA)).max() < 1e-9
    assert np.allclose(sb.pair_rr(e * 1e-12, A, ETA), np.eye(3) / (8 * np.pi * ETA * A ** 3), rtol=1e-9)


def test_grand_mobility_symmetric_positive_definite_with_overlaps():
    # two blobs at every separation from near coincidence to far
    for r in np.linspace(1e-3, 6 * A, 61):
        x = np.array([[0.0, 0.0, 0.0], [r * 0.6, r * 0.0, r * 0.8]])
        N = sb.grand_mobility(x, A, ETA)
        assert np.abs(N - N.T).max() < 1e-12 * np.abs(N).max()
        assert np.linalg.eigvalsh(N).min() > 0
    # a dense random cloud with many overlaps
    x = np.random.default_rng(2).uniform(0, 0.6, (40, 3))
    N = sb.grand_mobility(x, A, ETA)
    assert np.abs(N - N.T).max() < 1e-12 * np.abs(N).max()
    assert np.linalg.eigvalsh(N).min() > 0


def test_constrained_single_blob_solve_dense_equals_formal():
    w = W.chains_free_space(7, n_chains=2, bodies_per_chain=5)
    s = sb.SingleBlobSystem(w)
    U, phi = s.solve_dense()
    Uf, phif = s.solve_formal()
    C = s.S.C_dense()
    assert np.abs(U - Uf).max() < 1e-10 * np.abs(Uf).max()
    assert np.abs(C.T @ phi - C.T @ phif).max() < 1e-9 * np.abs(C.T @ phif).max()
    assert np.abs(C @ U - s.S.B_vec()).max() < 1e-12 * np.abs(U).max()


# Overlapping blobs: the integrand is singular on the circle where the two
# surfaces cross, so the quadrature converges slowly (about 5e-4 to 1.2e-3
# with 32 x 64 points per sphere at these separations, 1e-4 to 3e-4 with
# 48 x 96); 3e-3 still separates the closed forms from coefficients that
# keep continuity at contact and coincidence but are wrong
# (test_overlap_pin_rejects_contact_continuous_perturbations).
OVERLAP_QUAD = 3e-3


@pytest.mark.parametrize("r_over_a", [0.6, 1.2, 1.7])
def test_overlapping_rotational_pairs_equal_double_surface_averages(r_over_a):
    d = r_over_a * A * DIR
    Qrt, Qrr = rotational_averages(np.zeros(3), -d, A, ETA, 32, 64)
    Ert, Err = sb.pair_rt(d, A, ETA), sb.pair_rr(d, A, ETA)
    assert np.abs(Qrt - Ert).max() <= OVERLAP_QUAD * np.abs(Ert).max()
    assert np.abs(Qrr - Err).max() <= OVERLAP_QUAD * np.abs(Err).max()


def test_separated_rotational_pairs_equal_double_surface_averages():
    # beyond contact the integrand is smooth: the far forms to rounding
    for r_over_a in (2.5, 4.0):
        d = r_over_a * A * DIR
        Qrt, Qrr = rotational_averages(np.zeros(3), -d, A, ETA, 32, 64)
        assert np.abs(Qrt - sb.pair_rt(d, A, ETA)).max() <= 1e-10 * np.abs(Qrt).max()
        assert np.abs(Qrr - sb.pair_rr(d, A, ETA)).max() <= 1e-10 * np.abs(Qrr).max()


def test_overlap_pin_rejects_contact_continuous_perturbations():
    # Perturbed overlap coefficients that keep the values at r = 0 and at
    # r = 2a: rotation-from-torque I-coefficient 1 + (alpha + e) s + (beta -
    # e/4) s^3 (1 + 2 alpha + 8 beta fixed), rotation-from-force
    # (1 + e) s + (-3/8 - e/2) s^2 (2 alpha + 4 beta fixed), s = r/a, with a
    # coefficient change e = 1/32 (2.3 % and 8.4 % of the tensors at
    # r = 1.2a).  The quadrature must tell them apart by a wide margin.
    e = 1.0 / 32.0
    r_over_a = 1.2
    d = r_over_a * A * DIR
    s = r_over_a
    Qrt, Qrr = rotational_averages(np.zeros(3), -d, A, ETA, 32, 64)
    ee = np.outer(DIR, DIR)
    cI = 1 + (-27.0 / 32.0 + e) * s + (5.0 / 64.0 - e / 4) * s ** 3
    rr_bad = (cI * np.eye(3) + (9 * s / 32 - 3 * s ** 3 / 64) * ee) / (8 * np.pi * ETA * A ** 3)
    c = ((1 + e) * s - (3.0 / 8.0 + e / 2) * s * s) / (16 * np.pi * ETA * A * A)
    rt_bad = -c * sb.cross_matrix(DIR)
    assert np.abs(Qrr - rr_bad).max() > 5 * OVERLAP_QUAD * np.abs(Qrr).max()
    assert np.abs(Qrt - rt_bad).max() > 5 * OVERLAP_QUAD * np.abs(Qrt).max()
