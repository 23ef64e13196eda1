"""Pins of the steric-repulsion oracle: forces are minus the gradient of the
energy (finite differences), pair forces obey action and reaction (zero net
force and torque without a wall), pairs of the same articulated body and
beyond the cutoff do not interact, and the energy is continuous at contact."""
import numpy as np

from oracle import steric
from paper_2107_10800_gb300 import workloads as W

A, EPS, B, RC = 0.1, 0.3, 0.05, 0.6


def _blobs(seed=0, n_bodies=5, per=6, wall=0):
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.0, 1.2, (n_bodies * per, 3))
    if wall:
        r[:, 2] = rng.uniform(0.07, 0.6, len(r))
    off = np.arange(0, n_bodies * per + 1, per)
    assembly = np.array([0, 0, 1, 2, 3])[:n_bodies]
    return r, off, assembly


def test_forces_are_minus_the_energy_gradient():
    for wall in (0, 1):
        r, off, asm = _blobs(1, wall=wall)
        f = steric.blob_forces(r, off, asm, A, EPS, B, RC, wall, 0.2, 0.04)
        h = 1e-7
        for i in range(0, len(r), 5):
            for c in range(3):
                rp, rm = r.copy(), r.copy()
                rp[i, c] += h
                rm[i, c] -= h
                g = (steric.total_energy(rp, off, asm, A, EPS, B, RC, wall, 0.2, 0.04)
                     - steric.total_energy(rm, off, asm, A, EPS, B, RC, wall, 0.2, 0.04)) / (2 * h)
                assert abs(-g - f[i, c]) <= 1e-5 * max(1.0, abs(f[i, c]))


def test_action_reaction_and_exclusions():
    r, off, asm = _blobs(2)
    f = steric.blob_forces(r, off, asm, A, EPS, B, RC)
    assert np.abs(f.sum(axis=0)).max() < 1e-12
    assert np.abs(np.cross(r, f).sum(axis=0)).max() < 1e-12
    # one articulated body only: no pair forces
    f1 = steric.blob_forces(r, off, np.zeros(len(asm), int), A, EPS, B, RC)
    assert np.all(f1 == 0.0)
    # far apart beyond the cutoff: none either
    r2 = r.copy()
    r2[6:] += 100.0
    f2 = steric.blob_forces(r2[:12], off[:3], asm[:2], A, EPS, B, RC)
    assert np.all(f2[:6] == 0.0)


def test_energy_continuous_at_contact_and_body_sums():
    e_in = steric.pair_energy(2 * A - 1e-12, A, EPS, B)
    e_out = steric.pair_energy(2 * A + 1e-12, A, EPS, B)
    assert abs(e_in - e_out) < 1e-9 and abs(e_out - EPS) < 1e-9
    assert abs(steric.wall_energy(A, A, 0.2, 0.04) - 0.2) < 1e-15
    w = W.chains_free_space(1, n_chains=2, bodies_per_chain=2)
    r = w["q"][np.repeat(np.arange(4), 12)] + w["rho"]
    f = np.random.default_rng(3).standard_normal(r.shape)
    F = steric.body_forces(r, w["q"], w["blob_offset"], f)
    assert np.allclose(F[:, :3].sum(axis=0), f.sum(axis=0))
    # total torque about the origin = sum of body torques + q x body force
    tau = np.cross(r, f).sum(axis=0)
    assert np.allclose(F[:, 3:].sum(axis=0) + np.cross(w["q"], F[:, :3]).sum(axis=0), tau)
