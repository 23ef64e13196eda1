"""Single-blob bodies with rotational coupling (TEST INFRASTRUCTURE ONLY:
CPU oracle, FP64).

Sec. 2.4: a body can be one blob; then the body mobility N is the mobility of
the blobs including their rotational degrees of freedom (the generalised RPY
tensor), and the constrained problem is Eq. linear_system_general,
    U - N C^T phi = N F,    C U = B,
unknowns (U, phi), U = (u_p, omega_p) per body, F = (f_p, tau_p).

Generalised RPY tensor in free space for equal radii a, r = x_i - x_j,
r = |r|, e = r / r, mu0 = 1 / (6 pi eta a), [v]x w = v x w:
  translation-translation: the RPY tensor (oracle.mobility.rpy_free_pair)
  rotation from force (omega_i = M_rt F_j):
      r >= 2a:  -(1 / (8 pi eta r^2)) [e]x
      r <  2a:  -(1 / (16 pi eta a^2)) (r / a - 3 r^2 / (8 a^2)) [e]x
  translation from torque: M_tr(i, j) = M_rt(j, i)^T (= M_rt(i, j))
  rotation from torque:
      r >= 2a:  (1 / (16 pi eta r^3)) (3 e e^T - I)
      r <  2a:  (1 / (8 pi eta a^3)) [(1 - 27 r / (32 a) + 5 r^3 / (64 a^3)) I
                                      + (9 r / (32 a) - 3 r^3 / (64 a^3)) e e^T]
  self: mu0 I for translation, I / (8 pi eta a^3) for rotation, no coupling.
The far forms are the vorticity (half the curl) of the regularised
Stokeslet and of the rotlet, which the surface averages of Eq. RPY leave
unchanged (both are harmonic); the overlapping forms are the published
closed forms for equal spheres (Wajnryb, Mizerski, Zuk and Szymczak 2013).
Both are pinned by quadrature of the surface averages that define the
tensor (a force spread over the surface of one blob, a torque as the
surface density (3/(8 pi a^3)) T x n, the rotation of the other blob as
(3/(2a)) <n x u> over its surface), overlapping and separated.
"""
import numpy as np

from .mobility import rpy_free_pair
from .system import System


def cross_matrix(v):
    """[v]x with [v]x w = v x w."""
    v = np.asarray(v, float)
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def pair_rt(d, a, eta):
    """omega_i = M_rt F_j for separation d = x_i - x_j (d != 0)."""
    r = np.linalg.norm(d)
    e = np.asarray(d, float) / r
    if r >= 2 * a:
        c = 1.0 / (8 * np.pi * eta * r * r)
    else:
        c = (r / a - 3 * r * r / (8 * a * a)) / (16 * np.pi * eta * a * a)
    return -c * cross_matrix(e)


def pair_rr(d, a, eta):
    """omega_i = M_rr T_j for separation d = x_i - x_j (d != 0)."""
    r = np.linalg.norm(d)
    e = np.asarray(d, float) / r
    ee = np.outer(e, e)
    if r >= 2 * a:
        return (3 * ee - np.eye(3)) / (16 * np.pi * eta * r ** 3)
    s = r / a
    return ((1 - 27 * s / 32 + 5 * s ** 3 / 64) * np.eye(3)
            + (9 * s / 32 - 3 * s ** 3 / 64) * ee) / (8 * np.pi * eta * a ** 3)


def grand_mobility(x, a, eta):
    """Dense 6M x 6M mobility of single blobs at x (M, 3): rows and columns
    per blob ordered (u, omega) and (f, tau)."""
    x = np.asarray(x, float)
    M = len(x)
    N = np.zeros((6 * M, 6 * M))
    mu0 = 1.0 / (6 * np.pi * eta * a)
    mur = 1.0 / (8 * np.pi * eta * a ** 3)
    for i in range(M):
        N[6 * i:6 * i + 3, 6 * i:6 * i + 3] = mu0 * np.eye(3)
        N[6 * i + 3:6 * i + 6, 6 * i + 3:6 * i + 6] = mur * np.eye(3)
        for j in range(M):
            if i == j:
                continue
            d = x[i] - x[j]
            N[6 * i:6 * i + 3, 6 * j:6 * j + 3] = rpy_free_pair(d, a, eta)
            rt = pair_rt(d, a, eta)
            N[6 * i + 3:6 * i + 6, 6 * j:6 * j + 3] = rt
            N[6 * i:6 * i + 3, 6 * j + 3:6 * j + 6] = pair_rt(-d, a, eta).T
            N[6 * i + 3:6 * i + 6, 6 * j + 3:6 * j + 6] = pair_rr(d, a, eta)
    return N


class SingleBlobSystem:
    """Eq. linear_system_general for bodies that are single blobs (free
    space).  Links, C and B as for multiblob bodies (the workload's blobs,
    if any, are ignored: every body is one blob at its tracking point)."""

    def __init__(self, w, q=None, theta=None, dl=None, t=0.0):
        M = len(w["q"] if q is None else q)
        w1 = dict(w)
        w1["blob_offset"] = np.arange(M + 1)
        w1["rho"] = np.zeros((M, 3))
        self.S = System(w1, q=q, theta=theta, dl=dl, t=t)
        self.a = float(w["a"])
        self.eta = float(w["eta"])
        self.M_bodies = M
        self.P = self.S.P
        self.n = 6 * M + 3 * self.P

    def N_dense(self):
        return grand_mobility(self.S.q, self.a, self.eta)

    def rhs(self):
        """(N F, B)."""
        return np.concatenate([self.N_dense() @ self.S.F.ravel(), self.S.B_vec()])

    def A_dense(self):
        """[[I, -N C^T], [C, 0]] on (U, phi)."""
        N = self.N_dense()
        C = self.S.C_dense()
        M6, p3 = 6 * self.M_bodies, 3 * self.P
        A = np.zeros((self.n, self.n))
        A[:M6, :M6] = np.eye(M6)
        A[:M6, M6:] = -N @ C.T
        A[M6:, :M6] = C
        return A

    def solve_dense(self):
        y, *_ = np.linalg.lstsq(self.A_dense(), self.rhs(), rcond=None)
        return y[:6 * self.M_bodies], y[6 * self.M_bodies:]

    def solve_formal(self):
        """phi = (C N C^T)^+ (B - C N F), U = N (F + C^T phi)."""
        N = self.N_dense()
        C = self.S.C_dense()
        F = self.S.F.ravel()
        if self.P:
            phi = np.linalg.pinv(C @ N @ C.T, rcond=1e-12, hermitian=True) @ (self.S.B_vec() - C @ N @ F)
        else:
            phi = np.zeros(0)
        return N @ (F + C.T @ phi), phi


def euler_step(w, q, theta, t, dt, delta=1e-10, dl_now=None, dl_next=None):
    """One explicit Euler step (Sec. 4.3) of single-blob bodies: velocities
    from the dense solve, then the update, reconstruction and correction of
    the multiblob step.  Returns (q, theta, U)."""
    from .timestep import _stage_update
    sb = SingleBlobSystem(w, q=q, theta=theta, dl=dl_now, t=t)
    U, _ = sb.solve_dense()
    U = U.reshape(-1, 6)
    S = sb.S
    if dl_next is None:
        dl_next = w["dl"](t + dt)[:2] if w.get("dl") is not None else (S.dl_p, S.dl_q)
    q_n, th_n, _, _ = _stage_update(w, S.q, S.theta, U, S.assembly, S.bp, S.bq, dt, dl_next[0], dl_next[1],
                                    delta)
    return q_n, th_n, U
