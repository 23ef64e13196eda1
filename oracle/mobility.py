"""Blob mobility M (TEST INFRASTRUCTURE ONLY: CPU oracle).

Sec. 2.3, Eq. RPY: M_ij, which couples the force on blob j to the velocity of
blob i, is the double average of the Stokes Green's function over the
surfaces of the two blobs (radius a).  It is symmetric and positive definite
even for overlapping blobs.

Free space (Rotne-Prager-Yamakawa; the closed form of that double average for
equal radii, r = |r_i - r_j|, rhat = (r_i - r_j)/r, mu0 = 1/(6 pi eta a)):
    r >= 2a:  (1/(8 pi eta r)) [(1 + 2a^2/(3r^2)) I + (1 - 2a^2/r^2) rhat rhat]
    r <  2a:  mu0 [(1 - 9r/(32a)) I + (3r/(32a)) rhat rhat]
    r  = 0 :  mu0 I.

No-slip wall at z = 0 (Rotne-Prager-Blake): the free tensor above plus the
regularised image part of Blake's Green's function, generated symbolically by
gen_wall_image.py into wall_image.py.  Both blob centres must be higher than
a; the method is undefined otherwise.
"""
import numpy as np

from .wall_image import wall_image_8pieta


def rpy_free_pair(d, a, eta):
    """Free-space RPY tensor for separation vectors d = r_i - r_j.
    (..., 3) -> (..., 3, 3)."""
    d = np.asarray(d, dtype=np.float64)
    r = np.linalg.norm(d, axis=-1)
    mu0 = 1.0 / (6.0 * np.pi * eta * a)
    safe = np.where(r > 0, r, 1.0)
    rhat = d / safe[..., None]
    rr = rhat[..., :, None] * rhat[..., None, :]
    eye = np.broadcast_to(np.eye(3), rr.shape)
    far_c1 = (1.0 + 2.0 * a * a / (3.0 * safe ** 2)) / (8.0 * np.pi * eta * safe)
    far_c2 = (1.0 - 2.0 * a * a / safe ** 2) / (8.0 * np.pi * eta * safe)
    near_c1 = mu0 * (1.0 - 9.0 * r / (32.0 * a))
    near_c2 = mu0 * (3.0 * r / (32.0 * a))
    far = r >= 2.0 * a
    c1 = np.where(far, far_c1, near_c1)
    c2 = np.where(far, far_c2, near_c2)
    c2 = np.where(r > 0, c2, 0.0)
    return c1[..., None, None] * eye + c2[..., None, None] * rr


def rpy_wall_image_pair(ri, rj, a, eta):
    """Regularised image part of the wall mobility for targets ri and sources
    rj (both (..., 3)), divided by 8 pi eta."""
    ri = np.asarray(ri, dtype=np.float64)
    rj = np.asarray(rj, dtype=np.float64)
    Rx = ri[..., 0] - rj[..., 0]
    Ry = ri[..., 1] - rj[..., 1]
    Rz = ri[..., 2] + rj[..., 2]
    h = rj[..., 2] + 0.0 * ri[..., 2]
    return wall_image_8pieta(Rx, Ry, Rz, h, a) / (8.0 * np.pi * eta)


def pair_tensor(ri, rj, a, eta, wall):
    """M(r_i, r_j) for broadcast arrays of target and source positions."""
    M = rpy_free_pair(np.asarray(ri) - np.asarray(rj), a, eta)
    if wall:
        M = M + rpy_wall_image_pair(ri, rj, a, eta)
    return M


def _row_chunk(n, wall):
    """Target rows per vectorised block: bounds the temporaries of the
    generated wall expression (several hundred arrays of one block each)."""
    pairs = 100_000 if wall else 2_000_000
    return max(1, pairs // max(n, 1))


def check_heights(r, a):
    z = np.asarray(r)[:, 2]
    if np.any(z <= a):
        raise ValueError("blob centre at or below height a above the wall")


def mobility_dense(r, a, eta, wall):
    """Dense 3N x 3N mobility, block (i, j) = M(r_i, r_j)."""
    r = np.asarray(r, dtype=np.float64)
    n = len(r)
    if wall:
        check_heights(r, a)
    out = np.empty((n, 3, n, 3))
    chunk = _row_chunk(n, wall)
    for i0 in range(0, n, chunk):
        i1 = min(n, i0 + chunk)
        T = pair_tensor(r[i0:i1, None, :], r[None, :, :], a, eta, wall)
        out[i0:i1] = T.transpose(0, 2, 1, 3)
    return out.reshape(3 * n, 3 * n)


def mobility_rows(r, lam, rows, a, eta, wall):
    """u_i = sum_j M(r_i, r_j) lam_j for the target indices ``rows``
    (all sources).  Returns (len(rows), 3)."""
    r = np.asarray(r, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    rows = np.asarray(rows)
    if wall:
        check_heights(r, a)
    out = np.empty((len(rows), 3))
    chunk = _row_chunk(len(r), wall)
    for k0 in range(0, len(rows), chunk):
        idx = rows[k0:k0 + chunk]
        T = pair_tensor(r[idx, None, :], r[None, :, :], a, eta, wall)
        out[k0:k0 + chunk] = np.einsum("ijab,jb->ia", T, lam)
    return out


def mobility_matvec(r, lam, a, eta, wall):
    """u = M lam over all blobs."""
    return mobility_rows(r, lam, np.arange(len(r)), a, eta, wall)
