"""Pins of the periodic blob mobility oracle (oracle/periodic.py) against what
the mathematics fixes, independently of its own arithmetic:
  - the Ewald split is exact: the sum does not depend on xi;
  - the wave part's real-space transform W tends to the closed-form RPY
    tensor (mobility.rpy_free_pair, itself pinned by quadrature of the
    double surface average) as xi grows, overlaps and self term included;
  - the self-mobility of one blob in a cube of side L is
    mu0 [1 - c a/L + (4 pi/3)(a/L)^3] with c = 2.837297 (Hasimoto 1959,
    the Oseen lattice sum of a simple cubic array), exactly while 2a <= L;
  - periodicity, translation invariance, symmetry and positive definiteness;
  - the pair mobility tends to the free one as the box grows."""
import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import spherical_jn

from oracle import periodic as P
from oracle.mobility import rpy_free_pair

A, ETA = 0.1, 1.3
MU0 = 1.0 / (6.0 * np.pi * ETA * A)


def blobs(seed, n, box):
    rng = np.random.default_rng(seed)
    r = rng.random((n, 3)) * box
    r[1] = r[0] + [0.05, 0.1, 0.0]       # overlapping pair (r < 2a)
    r[2] = r[0] + [2.0 * A, 0.0, 0.0]    # pair at contact
    r[3] += [box[0], -2.0 * box[1], 0.0]  # centre outside the box
    return r


def test_split_parameter_independence():
    box = np.array([1.0, 1.2, 0.9])
    r = blobs(0, 12, box)
    Ms = [P.periodic_mobility_dense(r, A, ETA, box, xi) for xi in (4.0, 7.0, 13.0)]
    scale = np.abs(Ms[0]).max()
    for M in Ms[1:]:
        assert np.abs(M - Ms[0]).max() <= 1e-13 * scale


def test_wave_part_quadrature():
    # the composite Gauss-Legendre rule against an adaptive integrator
    xi = 9.0
    for r in (0.0, 0.07, 0.31):
        A_, B_ = P.wave_realspace_coefs(np.array([r]), A, xi)

        def f(k, which):
            base = P.hasimoto_split(k, xi) * np.sinc(k * A / np.pi) ** 2
            j0, j2 = spherical_jn(0, k * r), spherical_jn(2, k * r)
            return base * ((2.0 / 3.0) * j0 - j2 / 3.0 if which == 0 else j2)

        ka = quad(f, 0.0, 200.0, args=(0,), limit=400, epsabs=1e-14)[0] / (2 * np.pi ** 2)
        kb = quad(f, 0.0, 200.0, args=(1,), limit=400, epsabs=1e-14)[0] / (2 * np.pi ** 2)
        assert abs(A_[0] - ka) <= 1e-12 * abs(ka)
        assert abs(B_[0] - kb) <= 1e-12 * max(abs(kb), abs(ka))


def test_wave_part_tends_to_rpy():
    # beyond 2a the real-space remainder decays like exp(-xi^2 (r - 2a)^2)
    for d in ([0.4, 0.1, 0.1], [0.0, 0.0, 0.35], [0.2, 0.0, 0.1]):
        d = np.array(d)
        W = P.wave_realspace_tensor(d, A, ETA, 200.0)
        R = rpy_free_pair(d, A, ETA)
        assert np.abs(W - R).max() <= 1e-14 * MU0
    # overlapping: the remainder falls with xi (like 1/(xi a) at r = 0)
    for d in ([0.0, 0.0, 0.0], [0.03, 0.01, 0.0], [0.15, 0.05, 0.02]):
        d = np.array(d)
        R = rpy_free_pair(d, A, ETA)
        e1 = np.abs(P.wave_realspace_tensor(d, A, ETA, 200.0) - R).max()
        e2 = np.abs(P.wave_realspace_tensor(d, A, ETA, 400.0) - R).max()
        assert e2 <= 0.6 * e1 + 1e-15 * MU0
        assert e2 <= 4e-3 * MU0


@pytest.mark.parametrize("aL", [0.1, 0.2, 0.4])
def test_hasimoto_self_mobility(aL):
    L = A / aL
    M = P.periodic_mobility_dense(np.zeros((1, 3)), A, ETA, [L, L, L], 6.0 / L)
    assert np.abs(M - np.diag(np.diag(M))).max() <= 1e-15 * MU0  # isotropic
    m = M[0, 0] / MU0
    c = (1.0 - m + (4.0 * np.pi / 3.0) * aL ** 3) / aL
    assert abs(c - 2.837297) <= 1e-6
    # exact form: the same constant at every a/L
    assert abs(c - 2.8372974794806) <= 1e-11


def test_periodicity_translation_symmetry_definiteness():
    box = np.array([1.0, 1.2, 0.9])
    r = blobs(1, 10, box)
    M = P.periodic_mobility_dense(r, A, ETA, box, 6.0)
    r2 = r.copy()
    r2[5] += box * np.array([1, 0, -1])
    r3 = r + np.array([0.37, -0.21, 1.7])
    s = np.abs(M).max()
    assert np.abs(P.periodic_mobility_dense(r2, A, ETA, box, 6.0) - M).max() <= 1e-14 * s
    assert np.abs(P.periodic_mobility_dense(r3, A, ETA, box, 6.0) - M).max() <= 1e-14 * s
    assert np.abs(M - M.T).max() <= 1e-15 * s
    assert np.linalg.eigvalsh(M).min() > 0.0


def test_large_box_tends_to_free_space():
    # the box changes every pair by the same constant (the self shift) to
    # leading order; the rest falls like d^2 / L^3
    errs = []
    for d in ([0.3, 0.1, 0.0], [0.12, 0.0, 0.05]):
        d = np.array(d)
        e = []
        for L in (5.0, 10.0, 20.0):
            r = np.array([[0.0, 0.0, 0.0], d])
            M = P.periodic_mobility_dense(r, A, ETA, [L, L, L], 6.0 / L)
            pair = M[0:3, 3:6] - M[0:3, 0:3]
            free = rpy_free_pair(-d, A, ETA) - MU0 * np.eye(3)
            e.append(np.abs(pair - free).max() / MU0)
        errs.append(e)
    for e in errs:
        assert e[1] <= e[0] / 6.0 and e[2] <= e[1] / 6.0
        assert e[2] <= 1e-4
