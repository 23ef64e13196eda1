"""Time step with reconstruction and correction (TEST INFRASTRUCTURE ONLY:
CPU oracle).

Sec. 4.1: an articulated body a is tracked by its centre q_COM^a (mean of its
bodies' tracking points, Eq. ucom) and its bodies' orientations.  Positions
are rebuilt from g = P q + z(theta) = 0 (Eq. constraintCompact) with the
pseudo-inverse of the connectivity matrix:  q~^a = -(P^a)^+ z^a
(Eq. pseudo-inv-sol), q_p = q~_p + q_COM^a (Eq. reconst-up-COM).

Sec. 4.2: if ||g*||_2^2 >= delta after the update, the positions and
orientations are corrected by increments (dq_p, dtheta_p) minimising ||g||^2
subject to ||dtheta_p||^2 = 1 (Eq. min_probl_a/b, residual Eq. residual),
with the exact Jacobian (App. B).  The paper uses SciPy's trust-region least
squares; this oracle takes Levenberg-Marquardt steps on the residual
r = [g; ||dtheta_p||^2 - 1] from dq = 0, dtheta = [1, 0, 0, 0]:
    (J^T J + mu I) step = -J^T r,   mu = 1e-10 max diag(J^T J),
until ||r||^2 < delta^2.  Fixed damping rather than undamped minimum-norm
Gauss-Newton steps: link sets such as two links on a common axis leave
near-free directions (rotation about that axis) with singular values of J
down to ~1e-8, along which undamped steps move by orders of magnitude more
than the constraint violation; the damped step is the small correction, of
the size of the violation, that Sec. 4.2 describes.

Sec. 4.3 (explicit Euler with reconstruction and correction):
  U = solve(t_k); u_COM^a = mean_p u_p; q_COM* = q_COM + dt u_COM;
  theta* = theta_{omega dt} . theta; q* = reconstruct(theta*, t_{k+1});
  correct if ||g*||^2 >= delta.
"""
import numpy as np

from .kinematics import quat_mul, quat_from_rotvec, rotation_matrix
from .system import System


def assemblies_of(assembly, bp):
    """Map each articulated body to (bodies, links) index arrays."""
    out = {}
    link_asm = np.asarray(assembly)[np.asarray(bp)] if len(bp) else np.zeros(0, int)
    for a_ in np.unique(assembly):
        bodies = np.nonzero(assembly == a_)[0]
        links = np.nonzero(link_asm == a_)[0]
        out[int(a_)] = (bodies, links)
    return out


def connectivity_scalar(bodies, links, bp, bq):
    """P^a / I_3: the P_a x M_a incidence matrix, +1 at the link's body p and
    -1 at its body q (Eq. constraintCompact: g_n = q_p - q_q + z_n)."""
    col = {int(b): k for k, b in enumerate(bodies)}
    Ps = np.zeros((len(links), len(bodies)))
    for r_, n in enumerate(links):
        Ps[r_, col[int(bp[n])]] += 1.0
        Ps[r_, col[int(bq[n])]] -= 1.0
    return Ps


def z_vector(theta, dl_p, dl_q, bp, bq):
    """z_n = R(theta_p) dl_np - R(theta_q) dl_nq (Eq. constraintCompact)."""
    R = rotation_matrix(theta)
    return (np.einsum("nab,nb->na", R[bp], dl_p)
            - np.einsum("nab,nb->na", R[bq], dl_q))


def constraint_g(q, theta, dl_p, dl_q, bp, bq):
    """g_n = q_p + R_p dl_np - q_q - R_q dl_nq (Eq. constraint). (P, 3)."""
    return q[bp] - q[bq] + z_vector(theta, dl_p, dl_q, bp, bq)


def reconstruct(q_com, theta, dl_p, dl_q, assembly, bp, bq):
    """q_p = -( (P^a)^+ z^a )_p + q_COM^a for every body (Eq. pseudo-inv-sol
    and Eq. reconst-up-COM).  q_com: dict assembly -> (3,)."""
    z = z_vector(theta, dl_p, dl_q, bp, bq) if len(bp) else np.zeros((0, 3))
    q = np.zeros((len(theta), 3))
    for a_, (bodies, links) in assemblies_of(assembly, bp).items():
        if len(links):
            Ps = connectivity_scalar(bodies, links, bp, bq)
            qt = -np.linalg.pinv(Ps) @ z[links]
        else:
            qt = np.zeros((len(bodies), 3))
        q[bodies] = qt + q_com[a_]
    return q


def d_rot_apply(dth, v):
    """Derivatives of R(dtheta) v with respect to dtheta = [s, p] (from
    Eq. rot_mat): d/ds = 4 s v + 2 p x v,
    d/dp_l of component i = 2 delta_il (p . v) + 2 p_i v_l + 2 s eps_ilk v_k.
    Returns (3, 4)."""
    s, p = dth[0], dth[1:]
    J = np.zeros((3, 4))
    J[:, 0] = 4.0 * s * v + 2.0 * np.cross(p, v)
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1.0
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1.0
    J[:, 1:] = (2.0 * np.eye(3) * (p @ v) + 2.0 * np.outer(p, v)
                + 2.0 * s * np.einsum("ilk,k->il", eps, v))
    return J


def correction_residual(x, q, lt_p, lt_q, bp, bq, col):
    """Residual [g_n (Eq. residual); ||dtheta_p||^2 - 1] of one assembly.
    x holds (dq_p, dtheta_p) per body (7 per body); lt_* = R(theta) dl."""
    nb = len(col)
    X = x.reshape(nb, 7)
    g = []
    for k, n in enumerate(bp):
        p, qq = col[int(bp[k])], col[int(bq[k])]
        Rp = rotation_matrix(X[p, 3:])
        Rq = rotation_matrix(X[qq, 3:])
        g.append(q[k, 0] + X[p, :3] + Rp @ lt_p[k] - q[k, 1] - X[qq, :3] - Rq @ lt_q[k])
    unit = np.sum(X[:, 3:] ** 2, axis=1) - 1.0
    return np.concatenate([np.concatenate(g) if g else np.zeros(0), unit])


def correction_jacobian(x, lt_p, lt_q, bp, bq, col):
    """Exact Jacobian of correction_residual (App. B): for link n the 3 x 7
    blocks +[I, d(R(dth_p) l~_p)/d dth_p] on body p and
    -[I, d(R(dth_q) l~_q)/d dth_q] on body q; unit rows 2 dtheta_p^T."""
    nb = len(col)
    X = x.reshape(nb, 7)
    P = len(bp)
    J = np.zeros((3 * P + nb, 7 * nb))
    for k in range(P):
        p, qq = col[int(bp[k])], col[int(bq[k])]
        J[3 * k:3 * k + 3, 7 * p:7 * p + 3] += np.eye(3)
        J[3 * k:3 * k + 3, 7 * p + 3:7 * p + 7] += d_rot_apply(X[p, 3:], lt_p[k])
        J[3 * k:3 * k + 3, 7 * qq:7 * qq + 3] -= np.eye(3)
        J[3 * k:3 * k + 3, 7 * qq + 3:7 * qq + 7] -= d_rot_apply(X[qq, 3:], lt_q[k])
    for b in range(nb):
        J[3 * P + b, 7 * b + 3:7 * b + 7] = 2.0 * X[b, 3:]
    return J


def correct(q, theta, dl_p, dl_q, assembly, bp, bq, delta, max_iter=20):
    """Nonlinear correction (Sec. 4.2) of every articulated body whose
    constraint error is not yet below delta.  Returns (q, theta, iterations
    per assembly)."""
    q = q.copy()
    theta = theta.copy()
    R = rotation_matrix(theta)
    iters = {}
    for a_, (bodies, links) in assemblies_of(assembly, bp).items():
        if not len(links):
            continue
        col = {int(b): k for k, b in enumerate(bodies)}
        lbp, lbq = bp[links], bq[links]
        lt_p = np.einsum("nab,nb->na", R[lbp], dl_p[links])
        lt_q = np.einsum("nab,nb->na", R[lbq], dl_q[links])
        qpair = np.stack([q[lbp], q[lbq]], axis=1)
        x = np.zeros(7 * len(bodies))
        x.reshape(-1, 7)[:, 3] = 1.0
        it = 0
        while True:
            r = correction_residual(x, qpair, lt_p, lt_q, lbp, lbq, col)
            if r @ r < delta * delta or it >= max_iter:
                break
            J = correction_jacobian(x, lt_p, lt_q, lbp, lbq, col)
            N = J.T @ J
            mu = 1e-10 * np.diag(N).max()
            step = np.linalg.solve(N + mu * np.eye(len(N)), -J.T @ r)
            x = x + step
            it += 1
        iters[a_] = it
        X = x.reshape(-1, 7)
        q[bodies] = q[bodies] + X[:, :3]
        theta[bodies] = quat_mul(X[:, 3:], theta[bodies])
    return q, theta, iters


def euler_step(w, q, theta, t, dt, delta=1e-10, solve_tol=1e-12, x0=None,
               dl_now=None, dl_next=None):
    """One explicit Euler step of Sec. 4.3.  Returns (q, theta, info)."""
    S = System(w, q=q, theta=theta, dl=dl_now, t=t)
    b = S.rhs()
    if x0 is None:
        x0 = S.apply_preconditioner(b)
    y, its, hist = S.gmres(b=b, x0=x0, tol=solve_tol)
    lam, U, phi = S.split(y)
    U = U.reshape(-1, 6)
    assembly = S.assembly
    bp, bq = S.bp, S.bq
    # body-frame link vectors at t + dt
    if dl_next is not None:
        dlp1, dlq1 = dl_next[0], dl_next[1]
    elif w.get("dl") is not None:
        dlp1, dlq1 = w["dl"](t + dt)[:2]
    else:
        dlp1, dlq1 = S.dl_p, S.dl_q
    asm = assemblies_of(assembly, bp)
    q_com = {a_: q[bodies].mean(axis=0) + dt * U[bodies, :3].mean(axis=0)
             for a_, (bodies, _) in asm.items()}
    theta_s = quat_mul(quat_from_rotvec(U[:, 3:] * dt), theta)
    q_s = reconstruct(q_com, theta_s, dlp1, dlq1, assembly, bp, bq)
    g = constraint_g(q_s, theta_s, dlp1, dlq1, bp, bq) if len(bp) else np.zeros((0, 3))
    g2 = float(np.sum(g * g))
    corr_its = {}
    if g2 >= delta:
        q_n, th_n, corr_its = correct(q_s, theta_s, dlp1, dlq1, assembly, bp, bq, delta)
    else:
        q_n, th_n = q_s, theta_s
    g_after = constraint_g(q_n, th_n, dlp1, dlq1, bp, bq) if len(bp) else np.zeros((0, 3))
    info = dict(U=U, lam=lam, phi=phi, gmres_iters=its, residual=hist[-1],
                g2_before=g2, g2_after=float(np.sum(g_after * g_after)),
                corr_iters=corr_its, y=y, q_star=q_s, theta_star=theta_s)
    return q_n, th_n, info


def _stage_update(w, q0, theta0, U, assembly, bp, bq, h, dlp_end, dlq_end, delta):
    """Move the pose (q0, theta0) by h with body velocities U: each
    articulated body's centre by h times its mean body velocity (Eq. ucom),
    each orientation by theta_{omega h} . theta; reconstruct with the link
    vectors at the end (Eq. pseudo-inv-sol, reconst-up-COM) and correct when
    ||g*||^2 >= delta (Sec. 4.2).  Returns (q, theta, g2_before, g2_after)."""
    asm = assemblies_of(assembly, bp)
    q_com = {a_: q0[bodies].mean(axis=0) + h * U[bodies, :3].mean(axis=0)
             for a_, (bodies, _) in asm.items()}
    theta_s = quat_mul(quat_from_rotvec(U[:, 3:] * h), theta0)
    q_s = reconstruct(q_com, theta_s, dlp_end, dlq_end, assembly, bp, bq)
    g = constraint_g(q_s, theta_s, dlp_end, dlq_end, bp, bq) if len(bp) else np.zeros((0, 3))
    g2 = float(np.sum(g * g))
    if g2 >= delta:
        q_n, th_n, _ = correct(q_s, theta_s, dlp_end, dlq_end, assembly, bp, bq, delta)
    else:
        q_n, th_n = q_s, theta_s
    g_after = constraint_g(q_n, th_n, dlp_end, dlq_end, bp, bq) if len(bp) else np.zeros((0, 3))
    return q_n, th_n, g2, float(np.sum(g_after * g_after))


def midpoint_step(w, q, theta, t, dt, delta=1e-10, solve_tol=1e-12, dl_now=None, dl_half=None,
                  dl_next=None):
    """One explicit midpoint (RK2) step (App. "Midpoint scheme"): velocities
    at t; half step to the midpoint pose (reconstruction and correction with
    the link vectors at t + dt/2); velocities at the midpoint (links and
    their derivatives at t + dt/2); full step from the pose at t with the
    midpoint velocities, reconstruction and correction at t + dt.
    dl_half = (dlp, dlq, dlp_dot, dlq_dot) at t + dt/2 and dl_next = (dlp,
    dlq) at t + dt default to w["dl"] when the workload has time-dependent
    links and to the links at t otherwise.  Returns (q, theta, info)."""
    S = System(w, q=q, theta=theta, dl=dl_now, t=t)
    b = S.rhs()
    y0, its0, hist0 = S.gmres(b=b, x0=S.apply_preconditioner(b), tol=solve_tol)
    U0 = S.split(y0)[1].reshape(-1, 6)
    bp, bq, assembly = S.bp, S.bq, S.assembly
    if dl_half is None:
        dl_half = w["dl"](t + 0.5 * dt) if w.get("dl") is not None else (S.dl_p, S.dl_q, None, None)
    if dl_next is None:
        dl_next = w["dl"](t + dt)[:2] if w.get("dl") is not None else (S.dl_p, S.dl_q)
    q_h, th_h, g2h, _ = _stage_update(w, S.q, S.theta, U0, assembly, bp, bq, 0.5 * dt,
                                      dl_half[0], dl_half[1], delta)
    S2 = System(w, q=q_h, theta=th_h, dl=tuple(dl_half), t=t + 0.5 * dt)
    b2 = S2.rhs()
    y1, its1, hist1 = S2.gmres(b=b2, x0=S2.apply_preconditioner(b2), tol=solve_tol)
    lam1, U1, phi1 = S2.split(y1)
    U1 = U1.reshape(-1, 6)
    q_n, th_n, g2, g2a = _stage_update(w, S.q, S.theta, U1, assembly, bp, bq, dt, dl_next[0], dl_next[1],
                                       delta)
    info = dict(U=U1, lam=lam1, phi=phi1, U0=U0, q_half=q_h, theta_half=th_h, gmres_iters=its0 + its1,
                residual=max(hist0[-1], hist1[-1]), g2_before=g2, g2_after=g2a, g2_half=g2h, y=y1)
    return q_n, th_n, info
