"""Steric repulsion (TEST INFRASTRUCTURE ONLY: CPU oracle, FP64).

The paper adds a short-range repulsion between bacteria and between bacteria
and the wall to prevent overlaps (Sec. 5.3) without giving its form.  The
library's reading, which this module defines:
  between blobs i, j of different articulated bodies at distance r < r_c,
      U(r) = eps (1 + (2a - r) / b)      r <  2a
      U(r) = eps exp((2a - r) / b)       r >= 2a
  and, above a wall, on every blob at height h,
      U_w(h) = eps_w (1 + (a - h) / b_w)  h <  a
      U_w(h) = eps_w exp((a - h) / b_w)   h >= a
  (no cutoff for the wall term).  Blob forces are f = -grad U; a body
feels their sum and the sum of their torques about its tracking point,
K^T f (Sec. 2.3), added to its external force and torque.
"""
import numpy as np


def pair_energy(r, a, eps, b):
    r = np.asarray(r, float)
    return np.where(r < 2 * a, eps * (1.0 + (2 * a - r) / b), eps * np.exp((2 * a - r) / b))


def wall_energy(h, a, eps_w, b_w):
    h = np.asarray(h, float)
    return np.where(h < a, eps_w * (1.0 + (a - h) / b_w), eps_w * np.exp((a - h) / b_w))


def _assembly_of_blob(blob_offset, assembly):
    return np.repeat(np.asarray(assembly), np.diff(np.asarray(blob_offset)))


def total_energy(r, blob_offset, assembly, a, eps, b, rc, wall=0, eps_w=0.0, b_w=1.0):
    """Sum of the pair energies (each pair once) and the wall energies."""
    r = np.asarray(r, float)
    ab = _assembly_of_blob(blob_offset, assembly)
    d = np.linalg.norm(r[:, None, :] - r[None, :, :], axis=2)
    mask = (ab[:, None] != ab[None, :]) & (d < rc)
    E = 0.5 * np.sum(np.where(mask, pair_energy(d, a, eps, b), 0.0))
    if wall:
        E += np.sum(wall_energy(r[:, 2], a, eps_w, b_w))
    return E


def blob_forces(r, blob_offset, assembly, a, eps, b, rc, wall=0, eps_w=0.0, b_w=1.0):
    """f_i = -dU/dr_i (N, 3) by the analytic derivative of each term."""
    r = np.asarray(r, float)
    ab = _assembly_of_blob(blob_offset, assembly)
    n = len(r)
    f = np.zeros((n, 3))
    for i in range(n):
        d = r[i] - r
        dist = np.linalg.norm(d, axis=1)
        m = (ab != ab[i]) & (dist < rc) & (dist > 0)
        dd, rr = d[m], dist[m]
        # -dU/dr: eps / b inside 2a, eps / b exp((2a - r) / b) outside
        mag = np.where(rr < 2 * a, eps / b, eps / b * np.exp((2 * a - rr) / b))
        f[i] = np.sum((mag / rr)[:, None] * dd, axis=0)
    if wall:
        h = r[:, 2]
        f[:, 2] += np.where(h < a, eps_w / b_w, eps_w / b_w * np.exp((a - h) / b_w))
    return f


def body_forces(r, q, blob_offset, f):
    """K^T f: per body the sum of its blobs' forces and of their torques
    about the tracking point, (M, 6)."""
    off = np.asarray(blob_offset)
    out = np.zeros((len(off) - 1, 6))
    for p in range(len(off) - 1):
        s = slice(off[p], off[p + 1])
        out[p, :3] = f[s].sum(axis=0)
        out[p, 3:] = np.cross(r[s] - q[p], f[s]).sum(axis=0)
    return out
