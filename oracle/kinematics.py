"""Quaternion kinematics (TEST INFRASTRUCTURE ONLY: CPU oracle).

Sec. 2.1: theta = [s, p] is a unit quaternion; the rotation vector gamma has
quaternion [cos(gamma/2), sin(gamma/2) gamma/|gamma|] (Eq. after "fixed
axis"); the product of Eq. quaternion_mult composes rotations.
App. B, Eq. rot_mat: R(theta) = 2 [p p^T + s p^x + (s^2 - 1/2) I].
"""
import numpy as np


def quat_mul(t2, t1):
    """theta_2 . theta_1 (Eq. quaternion_mult): rotation t1 followed by t2.
    Works on (..., 4) arrays."""
    s2, p2 = t2[..., 0], t2[..., 1:]
    s1, p1 = t1[..., 0], t1[..., 1:]
    s = s2 * s1 - np.sum(p2 * p1, axis=-1)
    p = s2[..., None] * p1 + s1[..., None] * p2 + np.cross(p2, p1)
    return np.concatenate([s[..., None], p], axis=-1)


def quat_from_rotvec(gamma):
    """theta_gamma = [cos(g/2), sin(g/2) gamma/g], g = |gamma| (Sec. 2.1);
    the identity for gamma = 0.  (..., 3) -> (..., 4)."""
    gamma = np.asarray(gamma, dtype=np.float64)
    g = np.linalg.norm(gamma, axis=-1)
    out = np.zeros(gamma.shape[:-1] + (4,))
    out[..., 0] = np.cos(g / 2)
    safe = np.where(g > 0, g, 1.0)
    out[..., 1:] = (np.sin(g / 2) / safe)[..., None] * gamma
    out[..., 1:] = np.where((g > 0)[..., None], out[..., 1:], 0.0)
    return out


def cross_matrix(v):
    """v^x with v^x w = v x w.  (..., 3) -> (..., 3, 3)."""
    v = np.asarray(v, dtype=np.float64)
    z = np.zeros(v.shape[:-1])
    return np.stack([np.stack([z, -v[..., 2], v[..., 1]], -1),
                     np.stack([v[..., 2], z, -v[..., 0]], -1),
                     np.stack([-v[..., 1], v[..., 0], z], -1)], -2)


def rotation_matrix(theta):
    """R(theta) = 2 [p p^T + s p^x + (s^2 - 1/2) I] (App. B, Eq. rot_mat).
    (..., 4) -> (..., 3, 3)."""
    theta = np.asarray(theta, dtype=np.float64)
    s = theta[..., 0]
    p = theta[..., 1:]
    ppT = p[..., :, None] * p[..., None, :]
    eye = np.broadcast_to(np.eye(3), ppT.shape)
    return 2.0 * (ppT + s[..., None, None] * cross_matrix(p)
                  + (s * s - 0.5)[..., None, None] * eye)
