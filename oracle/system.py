"""Constrained mobility problem: operator, dense solution, preconditioner and
GMRES (TEST INFRASTRUCTURE ONLY: CPU oracle).

Unknowns y = (lambda, U, phi), ordered as in Eq. linear_system:
lambda (3 Nb) blob constraint forces, U (6 M) body velocities (u_p, omega_p),
phi (3 P) link Lagrange multipliers.

  A = [[ M,   -K,   0  ],        b = [ u_s, -F, B ]       (Eq. linear_system)
       [-K^T,  0,   C^T],
       [ 0,    C,   0  ]]

K: (K U)_i = u_p + omega_p x (r_i - q_p) for blob i of body p
   (Eq. no-slip-continuum, Eq. no-slip).
C: link n joining p and q, l_np = R(theta_p) dl_np, l_nq = R(theta_q) dl_nq;
   C_n U = u_p + omega_p x l_np - u_q - omega_q x l_nq (Eq. dg), i.e. the block
   row [I, -l_np^x, -I, l_nq^x] (App. A).
B_n = R(theta_q) d(dl_nq)/dt - R(theta_p) d(dl_np)/dt (Eq. dg).
"""
import numpy as np
import scipy.linalg as sla

from .kinematics import rotation_matrix, cross_matrix
from .mobility import mobility_dense


class System:
    """Dense FP64 representation of one configuration.

    w: workload dict (see paper_2107_10800_gb300.workloads); dl_p, dl_q are
    body-frame link vectors at the current time (or derived from w['joints']
    at the given pose), dlp_dot, dlq_dot their time derivatives (None =
    passive links)."""

    def __init__(self, w, q=None, theta=None, dl=None, t=0.0):
        self.eta = float(w["eta"])
        self.a = float(w["a"])
        self.wall = int(w["wall"])
        self.q = np.array(w["q"] if q is None else q, dtype=np.float64)
        self.theta = np.array(w["theta"] if theta is None else theta, dtype=np.float64)
        self.off = np.asarray(w["blob_offset"])
        self.rho = np.asarray(w["rho"], dtype=np.float64)
        self.F = np.asarray(w["F"], dtype=np.float64)
        self.assembly = np.asarray(w["assembly"])
        self.bp = np.asarray(w["body_p"])
        self.bq = np.asarray(w["body_q"])
        self.M_bodies = len(self.q)
        self.P = len(self.bp)
        self.Nb = int(self.off[-1])
        self.body_of_blob = np.repeat(np.arange(self.M_bodies), np.diff(self.off))
        self.R = rotation_matrix(self.theta)
        # Lab-frame blob positions r_i = q_p + R(theta_p) rho_i (Sec. 2.3).
        self.r = self.q[self.body_of_blob] + np.einsum(
            "nab,nb->na", self.R[self.body_of_blob], self.rho)
        if dl is not None:
            self.dl_p, self.dl_q, self.dlp_dot, self.dlq_dot = [
                None if v is None else np.asarray(v, dtype=np.float64) for v in dl]
        elif w.get("dl") is not None:
            self.dl_p, self.dl_q, self.dlp_dot, self.dlq_dot = w["dl"](t)
        elif self.P > 0:
            self.dl_p, self.dl_q = joints_to_body_frame(
                w["joints"], self.q, self.R, self.bp, self.bq)
            self.dlp_dot = self.dlq_dot = None
        else:
            self.dl_p = self.dl_q = np.zeros((0, 3))
            self.dlp_dot = self.dlq_dot = None
        self.n = 3 * self.Nb + 6 * self.M_bodies + 3 * self.P

    # ----- pieces of the operator -------------------------------------
    def l_lab(self):
        """l_np = R_p dl_np and l_nq = R_q dl_nq (lab frame)."""
        lp = np.einsum("nab,nb->na", self.R[self.bp], self.dl_p)
        lq = np.einsum("nab,nb->na", self.R[self.bq], self.dl_q)
        return lp, lq

    def K_dense(self):
        """3Nb x 6M matrix of Eq. no-slip: blob rows [I, -(r_i - q_p)^x]."""
        K = np.zeros((3 * self.Nb, 6 * self.M_bodies))
        for i in range(self.Nb):
            p = self.body_of_blob[i]
            K[3 * i:3 * i + 3, 6 * p:6 * p + 3] = np.eye(3)
            K[3 * i:3 * i + 3, 6 * p + 3:6 * p + 6] = -cross_matrix(self.r[i] - self.q[p])
        return K

    def C_dense(self):
        """3P x 6M constraint Jacobian (Eq. dg, App. A)."""
        C = np.zeros((3 * self.P, 6 * self.M_bodies))
        lp, lq = self.l_lab()
        for n in range(self.P):
            p, q = self.bp[n], self.bq[n]
            C[3 * n:3 * n + 3, 6 * p:6 * p + 3] += np.eye(3)
            C[3 * n:3 * n + 3, 6 * p + 3:6 * p + 6] += -cross_matrix(lp[n])
            C[3 * n:3 * n + 3, 6 * q:6 * q + 3] += -np.eye(3)
            C[3 * n:3 * n + 3, 6 * q + 3:6 * q + 6] += cross_matrix(lq[n])
        return C

    def B_vec(self):
        """B_n = R_q d(dl_nq)/dt - R_p d(dl_np)/dt; zero for passive links."""
        if self.dlp_dot is None:
            return np.zeros(3 * self.P)
        bq = np.einsum("nab,nb->na", self.R[self.bq], self.dlq_dot)
        bp = np.einsum("nab,nb->na", self.R[self.bp], self.dlp_dot)
        return (bq - bp).ravel()

    def mobility(self):
        if not hasattr(self, "_M"):
            self._M = mobility_dense(self.r, self.a, self.eta, self.wall)
        return self._M

    def A_dense(self):
        """The saddle-point matrix of Eq. linear_system."""
        Mm = self.mobility()
        K = self.K_dense()
        C = self.C_dense()
        nl, nu, nf = 3 * self.Nb, 6 * self.M_bodies, 3 * self.P
        A = np.zeros((self.n, self.n))
        A[:nl, :nl] = Mm
        A[:nl, nl:nl + nu] = -K
        A[nl:nl + nu, :nl] = -K.T
        A[nl:nl + nu, nl + nu:] = C.T
        A[nl + nu:, nl:nl + nu] = C
        return A

    def rhs(self, u_s=None):
        """b = (u_s, -F, B) (Eq. linear_system)."""
        us = np.zeros(3 * self.Nb) if u_s is None else np.asarray(u_s).ravel()
        return np.concatenate([us, -self.F.ravel(), self.B_vec()])

    def split(self, y):
        nl, nu = 3 * self.Nb, 6 * self.M_bodies
        return y[:nl], y[nl:nl + nu], y[nl + nu:]

    # ----- solutions -----------------------------------------------------
    def solve_dense(self, b=None):
        """Exact solution of A y = b by a dense least-squares solve (A is
        singular when C lacks full row rank; the minimum-norm solution is
        returned then)."""
        b = self.rhs() if b is None else b
        A = self.A_dense()
        y, *_ = sla.lstsq(A, b, lapack_driver="gelsy", cond=1e-13)
        return y

    def solve_formal(self, b=None):
        """Solution through the body mobility N = (K^T M^-1 K)^-1 and the
        constraint resistance G = (C N C^T)^+ (Eq. U and the formula for
        U-hat after Eq. linear_system):  U = U-hat + N C^T phi,
        phi = G (B - C U-hat), U-hat = N F - N K^T M^-1 u_s (with the
        right-hand side b = (u_s, -F, B) read off b), lambda = M^-1 (u_s + K U).
        An independent route to the same (lambda, U, C^T phi)."""
        b = self.rhs() if b is None else b
        us, mF, Bv = self.split(b)
        Mm = self.mobility()
        K = self.K_dense()
        C = self.C_dense()
        cf = sla.cho_factor(Mm)
        MinvK = sla.cho_solve(cf, K)
        Minv_us = sla.cho_solve(cf, us)
        N = np.linalg.inv(K.T @ MinvK)
        Uhat = N @ (-mF) - N @ (K.T @ Minv_us)
        if self.P:
            G = np.linalg.pinv(C @ N @ C.T, rcond=1e-12, hermitian=True)
            phi = G @ (Bv - C @ Uhat)
            U = Uhat + N @ (C.T @ phi)
        else:
            phi = np.zeros(0)
            U = Uhat
        lam = sla.cho_solve(cf, us + K @ U)
        return np.concatenate([lam, U, phi])

    # ----- block-diagonal preconditioner (Sec. 3.1) ---------------------
    def build_preconditioner(self):
        """M-tilde = blockdiag_p M^(pp) (blobs of the same body only);
        N-tilde_p = [(K^(p))^T (M^(pp))^-1 K^(p)]^-1 per body (Eq. for N-tilde,
        read with the inverse on M^(pp) as for N in Sec. 2.3);
        G-tilde_a = [C^(a) N-tilde^(aa) (C^(a))^T]^+ per articulated body
        (Eq. block_diag_const_res; pseudo-inverse when C lacks full row rank)."""
        Mm = self.mobility()
        K = self.K_dense()
        C = self.C_dense()
        self._pc_Minv = []
        self._pc_N = []
        for p in range(self.M_bodies):
            s = slice(3 * self.off[p], 3 * self.off[p + 1])
            Mpp = Mm[s, s]
            Kp = K[s, 6 * p:6 * p + 6]
            Minv = np.linalg.inv(Mpp)
            self._pc_Minv.append(Minv)
            self._pc_N.append(np.linalg.inv(Kp.T @ Minv @ Kp))
        Nt = sla.block_diag(*self._pc_N) if self.M_bodies else np.zeros((0, 0))
        self._pc_G = {}
        link_assembly = self.assembly[self.bp]
        for a_ in np.unique(link_assembly):
            links = np.nonzero(link_assembly == a_)[0]
            rows = np.concatenate([np.arange(3 * n, 3 * n + 3) for n in links])
            Ca = C[rows]
            H = Ca @ Nt @ Ca.T
            self._pc_G[a_] = (rows, np.linalg.pinv(H, rcond=1e-12, hermitian=True))
        self._pc_K = K
        self._pc_C = C
        self._pc_Nt = Nt

    def apply_preconditioner(self, r):
        """Exact solution of the block-diagonal approximate problem
        (Eq. precond) for the right-hand side r = (r1, r2, r3):
          rows 1-2 give  U = U-hat + N-tilde C^T phi,
                         U-hat = N-tilde (-r2 - K^T M-tilde^-1 r1);
          row 3 gives    phi = G-tilde (r3 - C U-hat);
          row 1 gives    lambda = M-tilde^-1 (r1 + K U)."""
        if not hasattr(self, "_pc_N"):
            self.build_preconditioner()
        r1, r2, r3 = self.split(np.asarray(r, dtype=np.float64))
        K, C, Nt = self._pc_K, self._pc_C, self._pc_Nt
        w = np.zeros_like(r1)
        for p in range(self.M_bodies):
            s = slice(3 * self.off[p], 3 * self.off[p + 1])
            w[s] = self._pc_Minv[p] @ r1[s]
        Uhat = Nt @ (-r2 - K.T @ w)
        phi = np.zeros(3 * self.P)
        c = r3 - C @ Uhat
        for rows, G in self._pc_G.values():
            phi[rows] = G @ c[rows]
        U = Uhat + Nt @ (C.T @ phi)
        lam = np.zeros_like(r1)
        t = r1 + K @ U
        for p in range(self.M_bodies):
            s = slice(3 * self.off[p], 3 * self.off[p + 1])
            lam[s] = self._pc_Minv[p] @ t[s]
        return np.concatenate([lam, U, phi])

    def apply_A(self, y):
        """A y with the dense mobility."""
        lam, U, phi = self.split(np.asarray(y, dtype=np.float64))
        K, C = self.K_dense(), self.C_dense()
        return np.concatenate([self.mobility() @ lam - K @ U,
                               -K.T @ lam + C.T @ phi,
                               C @ U])

    def gmres(self, b=None, x0=None, tol=1e-10, restart=50, max_iter=500):
        """Right-preconditioned restarted GMRES with modified Gram-Schmidt
        (Sec. 3.1 uses preconditioned GMRES; right preconditioning makes the
        minimised residual the true one).  Stops when
        ||b - A y||_2 / ||b||_2 <= tol.  Returns (y, iterations, history)."""
        b = self.rhs() if b is None else np.asarray(b, dtype=np.float64)
        return gmres_right(self.apply_A, self.apply_preconditioner, b,
                           x0=x0, tol=tol, restart=restart, max_iter=max_iter)


def joints_to_body_frame(joints, q, R, bp, bq):
    """Body-frame link vectors of passive links from their lab-frame joint
    points at the current pose: dl_np = R_p^T (j_n - q_p), dl_nq likewise, so
    that g_n = 0 (Eq. constraint)."""
    joints = np.asarray(joints, dtype=np.float64)
    dl_p = np.einsum("nba,nb->na", R[bp], joints - q[bp])
    dl_q = np.einsum("nba,nb->na", R[bq], joints - q[bq])
    return dl_p, dl_q


def gmres_right(apply_A, apply_P, b, x0=None, tol=1e-10, restart=50, max_iter=500):
    """Textbook restarted GMRES(m) on A P^-1 z = b, y = x0 + P^-1 V xi, with
    modified Gram-Schmidt and Givens rotations."""
    n = len(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n), 0, [0.0]
    hist = []
    it = 0
    while True:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta / bnorm <= tol or it >= max_iter:
            return x, it, hist
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k_done = 0
        for j in range(restart):
            w = apply_A(apply_P(V[j]))
            for i in range(j + 1):
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol or it >= max_iter:
                break
        xi = sla.solve_triangular(H[:k_done, :k_done], g[:k_done])
        x = x + apply_P(V[:k_done].T @ xi)
