"""Sphere quadrature for checking the blob mobility against its definition
(Sec. 2.3, Eq. RPY: the double average of a Green's function over two blob
surfaces).  Gauss-Legendre in cos(polar angle) times the midpoint rule in the
azimuth; weights normalised to one, so sums are surface averages."""
import numpy as np


def sphere_rule(nt, nphi):
    x, w = np.polynomial.legendre.leggauss(nt)
    ph = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    X, P = np.meshgrid(x, ph, indexing="ij")
    st = np.sqrt(1 - X ** 2)
    pts = np.stack([st * np.cos(P), st * np.sin(P), X], -1).reshape(-1, 3)
    wts = np.repeat(w, nphi) / (2 * nphi)
    return pts, wts


def oseen(x, y, eta):
    """Free-space Green's function (Oseen tensor) G_ij(x, y)/(8 pi eta)."""
    d = x - y
    r = np.linalg.norm(d, axis=-1)
    return (np.eye(3) / r[..., None, None]
            + d[..., :, None] * d[..., None, :] / r[..., None, None] ** 3) / (8 * np.pi * eta)


def blake(x, y, eta):
    """Blake's Green's function of a point force at y above the no-slip plane
    z = 0, evaluated at x (Blake 1971): Oseen(x - y) - Oseen(x - y*) plus the
    Stokes-doublet and source-dipole images, written out term by term:
      2 h D_jj d/dR_j [ h R_i/R^3 - delta_i3/R - R_i R_3/R^3 ],  R = x - y*,
    D = diag(1, 1, -1), h = y_3."""
    x = np.asarray(x, float)
    y = np.asarray(y, float)
    ys = y * np.array([1.0, 1.0, -1.0])
    R = x - ys
    Rn = np.linalg.norm(R, axis=-1)[..., None, None]
    h = (y[..., 2] + 0 * x[..., 2])[..., None, None]
    Ri = R[..., :, None]
    Rj = R[..., None, :]
    e3i = np.array([0.0, 0.0, 1.0])[:, None]
    e3j = np.array([0.0, 0.0, 1.0])[None, :]
    I = np.eye(3)
    R3 = R[..., 2][..., None, None]
    # d/dR_j of the bracket, component i
    d_hRi = h * (I / Rn ** 3 - 3 * Ri * Rj / Rn ** 5)
    d_e3 = -e3i * (-Rj / Rn ** 3)
    d_RiR3 = -(I * R3 / Rn ** 3 + Ri * e3j / Rn ** 3 - 3 * Ri * R3 * Rj / Rn ** 5)
    D = np.array([1.0, 1.0, -1.0])[None, :]
    img = 2 * h * D * (d_hRi + d_e3 + d_RiR3)
    G = oseen(x, y, eta) * 8 * np.pi * eta - (I / Rn + Ri * Rj / Rn ** 3) + img
    return G / (8 * np.pi * eta)


def double_average(G, xi, xj, a, eta, nt, nphi):
    """(1/(4 pi a^2))^2 double surface integral of G over the spheres of
    radius a about xi (first argument) and xj (second argument)."""
    pts, w = sphere_rule(nt, nphi)
    A = xi + a * pts
    B = xj + a * pts
    out = np.zeros((3, 3))
    for k in range(len(A)):
        out += w[k] * np.einsum("j,jab->ab", w, G(A[k][None, :], B, eta))
    return out


def _cross_matrices(n):
    """[n_k]x for each row n_k (so that [n]x v = n x v)."""
    Z = np.zeros((len(n), 3, 3))
    Z[:, 0, 1], Z[:, 0, 2] = -n[:, 2], n[:, 1]
    Z[:, 1, 0], Z[:, 1, 2] = n[:, 2], -n[:, 0]
    Z[:, 2, 0], Z[:, 2, 1] = -n[:, 1], n[:, 0]
    return Z


def rotational_averages(xi, xj, a, eta, nt, nphi):
    """Rotation-from-force and rotation-from-torque couplings of two blobs of
    radius a about xi (rotating) and xj (forced), by the surface averages
    that define the generalised RPY tensor (Sec. 2.4: a force F_j spread
    evenly over the surface of blob j, a torque T_j as the surface force
    density (3/(8 pi a^3)) T_j x n; the rotation of blob i as the rigid
    rotation fitted to the flow on its surface, (3/(2a)) <n x u>_{S_i}, which
    returns omega for u = omega x (x - xi)):
        M_rt = (3/(2a)) < [n_x]x <G(x, y)>_y >_x
        M_rr = -(3/(2a))^2 < [n_x]x <G(x, y) [n_y]x>_y >_x
    with G the Oseen tensor.  Returns (M_rt, M_rr)."""
    pts, w = sphere_rule(nt, nphi)
    X = _cross_matrices(pts)
    A = xi + a * pts
    B = xj + a * pts
    rt = np.zeros((3, 3))
    rr = np.zeros((3, 3))
    for k in range(len(A)):
        G = oseen(A[k][None, :], B, eta)
        rt += w[k] * X[k] @ np.einsum("j,jab->ab", w, G)
        rr += w[k] * X[k] @ np.einsum("j,jab,jbc->ac", w, G, X)
    c = 3.0 / (2.0 * a)
    return c * rt, -c * c * rr
