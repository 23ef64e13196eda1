"""Periodic blob mobility (TEST INFRASTRUCTURE ONLY: CPU oracle).

The suspensions of Sec. 5.3 are also run with periodic boundary conditions.
This module gives the blob mobility of a triply periodic box
[0, Lx) x [0, Ly) x [0, Lz) (volume V) with zero mean flow, for the free-space
RPY tensor of Sec. 2.3 (Eq. RPY: the Oseen tensor averaged over the surfaces
of both blobs).

Definition.  In Fourier space the Oseen tensor is (I - khat khat) / (eta k^2)
and each surface average of radius a multiplies it by sinc(ka) =
sin(ka) / (ka), so the periodic RPY mobility is the lattice sum
    M_per(d) = 1/(eta V) sum_{k != 0} sinc^2(ka) (I - khat khat) / k^2 e^{i k.d},
    k = 2 pi (m_x / Lx, m_y / Ly, m_z / Lz),  m integer,
for every pair, the self pair (d = 0) included.  The k = 0 term is left out:
the mean flow over the box is zero (the net force on the fluid is balanced
by the mean pressure gradient).

Evaluation (Ewald's split; the splitting function is Hasimoto's,
H(k) = (1 + k^2/(4 xi^2)) exp(-k^2/(4 xi^2)), xi > 0 free):
    M_per(d) = sum_n [M_RPY(d + n) - W(d + n)] + wave(d)
    wave(d)  = 1/(eta V) sum_{k != 0} H(k) sinc^2(ka) (I - khat khat)/k^2 e^{i k.d}
    W(r)     = the inverse Fourier transform over R^3 of the wave multiplier,
             = 1/(2 pi^2 eta) int_0^inf H sinc^2(ka)
                   [(2/3) j0(kr) I + j2(kr) (rhat rhat - I/3)] dk
with n over the lattice vectors (n_x Lx, n_y Ly, n_z Lz) and M_RPY the closed
form of mobility.rpy_free_pair.  M_RPY - W is the inverse transform of the
multiplier times 1 - H = O(k^4): it decays like exp(-xi^2 (r - 2a)^2), so
the image sum is cut at r = 2a + 7/xi; the wave sum is cut at |k| =
2 xi sqrt(50), beyond which H < 1e-20.  The result does not depend on xi;
tests/test_oracle_periodic.py pins it by that independence, by the limit
xi -> inf of W (which must give M_RPY, overlaps and self term included), by
Hasimoto's self-mobility constant of a cubic lattice, by periodicity and by
positive definiteness.
"""
import numpy as np
from scipy.special import spherical_jn

from .mobility import rpy_free_pair


def hasimoto_split(k, xi):
    """H(k) = (1 + k^2/(4 xi^2)) exp(-k^2/(4 xi^2))."""
    x = (np.asarray(k, dtype=np.float64) / (2.0 * xi)) ** 2
    return (1.0 + x) * np.exp(-x)


def _sinc(x):
    return np.sinc(np.asarray(x) / np.pi)  # numpy's sinc is sin(pi x)/(pi x)


def _gauss_legendre(k_max, periods):
    """Composite 20-point Gauss-Legendre nodes and weights on [0, k_max] with
    at least 4 panels per oscillation period of the integrand."""
    panels = int(max(64, np.ceil(4 * periods)))
    x, w = np.polynomial.legendre.leggauss(20)
    edges = np.linspace(0.0, k_max, panels + 1)
    half = 0.5 * np.diff(edges)
    mid = 0.5 * (edges[1:] + edges[:-1])
    nodes = (mid[:, None] + half[:, None] * x[None, :]).ravel()
    weights = (half[:, None] * w[None, :]).ravel()
    return nodes, weights


def wave_realspace_coefs(r, a, xi):
    """Scalars (A, B) with W(r) = (A I + B rhat rhat) / eta for distances r
    (any shape):
        A = 1/(2 pi^2) int H sinc^2(ka) [(2/3) j0(kr) - j2(kr)/3] dk
        B = 1/(2 pi^2) int H sinc^2(ka) j2(kr) dk."""
    r = np.asarray(r, dtype=np.float64)
    k_max = 2.0 * xi * np.sqrt(50.0)
    span = max(float(np.max(r)) if r.size else 0.0, 2.0 * a)
    k, wk = _gauss_legendre(k_max, k_max * span / (2.0 * np.pi))
    base = hasimoto_split(k, xi) * _sinc(k * a) ** 2 * wk
    flat = r.ravel()
    A = np.empty(flat.shape)
    B = np.empty(flat.shape)
    for s in range(0, len(flat), 256):
        kr = flat[s:s + 256, None] * k[None, :]
        j0 = spherical_jn(0, kr)
        j2 = spherical_jn(2, kr)
        A[s:s + 256] = ((2.0 / 3.0) * j0 - j2 / 3.0) @ base
        B[s:s + 256] = j2 @ base
    c = 1.0 / (2.0 * np.pi ** 2)
    return (c * A).reshape(r.shape), (c * B).reshape(r.shape)


def wave_realspace_tensor(d, a, eta, xi):
    """W(d) for separation vectors d (..., 3) -> (..., 3, 3)."""
    d = np.asarray(d, dtype=np.float64)
    r = np.linalg.norm(d, axis=-1)
    A, B = wave_realspace_coefs(r, a, xi)
    safe = np.where(r > 0, r, 1.0)
    rhat = d / safe[..., None]
    rr = rhat[..., :, None] * rhat[..., None, :]
    return (A[..., None, None] * np.eye(3) + B[..., None, None] * rr) / eta


def _images(box, r_cut):
    """Lattice vectors n with |n_d| <= r_cut + L_d (enough for differences
    already wrapped into [-L/2, L/2))."""
    box = np.asarray(box, dtype=np.float64)
    nmax = np.ceil(r_cut / box).astype(int) + 1
    rng = [np.arange(-m, m + 1) for m in nmax]
    n = np.stack(np.meshgrid(*rng, indexing="ij"), axis=-1).reshape(-1, 3)
    return n * box


def _kvectors(box, xi):
    """Nonzero wave vectors 2 pi m / L with |k| <= 2 xi sqrt(50)."""
    box = np.asarray(box, dtype=np.float64)
    k_max = 2.0 * xi * np.sqrt(50.0)
    mmax = np.floor(k_max * box / (2.0 * np.pi)).astype(int)
    rng = [np.arange(-m, m + 1) for m in mmax]
    m = np.stack(np.meshgrid(*rng, indexing="ij"), axis=-1).reshape(-1, 3)
    k = 2.0 * np.pi * m / box
    k2 = np.sum(k * k, axis=1)
    keep = (k2 > 0) & (k2 <= k_max ** 2)
    return k[keep]


def periodic_mobility_dense(r, a, eta, box, xi=None):
    """Dense 3N x 3N periodic mobility; block (i, j) = M_per(r_i - r_j)."""
    r = np.asarray(r, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    n = len(r)
    if xi is None:
        xi = 6.0 / float(np.min(box))
    V = float(np.prod(box))
    # real space: all pairs, all images within the cut
    r_cut = 2.0 * a + 7.0 / xi
    d = r[:, None, :] - r[None, :, :]
    d = d - box * np.round(d / box)
    out = np.zeros((n, n, 3, 3))
    for nv in _images(box, r_cut):
        e = d + nv
        dist = np.linalg.norm(e, axis=-1)
        near = dist < r_cut
        if not np.any(near):
            continue
        ii, jj = np.nonzero(near)
        ev = e[ii, jj]
        out[ii, jj] += rpy_free_pair(ev, a, eta) - wave_realspace_tensor(ev, a, eta, xi)
    # wave space: sum over k of S(k) cos(k . (r_i - r_j))
    k = _kvectors(box, xi)
    k2 = np.sum(k * k, axis=1)
    khat = k / np.sqrt(k2)[:, None]
    scal = hasimoto_split(np.sqrt(k2), xi) * _sinc(np.sqrt(k2) * a) ** 2 / (k2 * eta * V)
    proj = np.eye(3)[None] - khat[:, :, None] * khat[:, None, :]
    Sk = scal[:, None, None] * proj  # (nk, 3, 3)
    for s in range(0, len(k), 4096):
        ks = k[s:s + 4096]
        ph = r @ ks.T
        C, Sn = np.cos(ph), np.sin(ph)
        T = Sk[s:s + 4096]
        for a_ in range(3):
            for b_ in range(3):
                w_ = T[:, a_, b_]
                out[:, :, a_, b_] += (C * w_) @ C.T + (Sn * w_) @ Sn.T
    return out.transpose(0, 2, 1, 3).reshape(3 * n, 3 * n)


def periodic_mobility_matvec(r, lam, a, eta, box, xi=None):
    """u = M_per lam (small N only: forms the dense matrix)."""
    Mp = periodic_mobility_dense(r, a, eta, box, xi)
    return (Mp @ np.asarray(lam, dtype=np.float64).ravel()).reshape(-1, 3)
