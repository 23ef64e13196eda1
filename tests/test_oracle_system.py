"""Pins of the oracle's constrained mobility problem (Sec. 2.2-3.1, App. A):
finite differences of the holonomic constraint and of the blob positions,
symmetry, two independent solution routes, conservation properties, the
projection property and the preconditioner's defining equation."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.system import System
from oracle.kinematics import quat_mul, quat_from_rotvec, rotation_matrix
from oracle.timestep import constraint_g
from paper_2107_10800_gb300 import workloads


@pytest.fixture(scope="module")
def chains():
    return workloads.chains_free_space(1)


@pytest.fixture(scope="module")
def chains_sys(chains):
    return System(chains)


def small_colony(seed=2):
    # 6 rods of 2x8 blobs: same link pattern as the colony workload, small.
    return workloads.diatom_colony(seed, n_rods=6, nx=8)


def test_K_is_rigid_motion_derivative(chains_sys):
    # (K U)_i = d r_i / dt for the motion dq/dt = u, dtheta/dt = 1/2 [0, w] . theta.
    S = chains_sys
    rng = np.random.default_rng(0)
    U = rng.standard_normal((S.M_bodies, 6))
    eps = 1e-6
    rr = []
    for sgn in (1, -1):
        q = S.q + sgn * eps * U[:, :3]
        th = quat_mul(quat_from_rotvec(sgn * eps * U[:, 3:]), S.theta)
        R = rotation_matrix(th)
        rr.append(q[S.body_of_blob] + np.einsum("nab,nb->na", R[S.body_of_blob], S.rho))
    fd = (rr[0] - rr[1]) / (2 * eps)
    KU = (S.K_dense() @ U.ravel()).reshape(-1, 3)
    assert np.abs(fd - KU).max() <= 1e-8 * np.abs(KU).max()


def test_C_and_B_are_constraint_time_derivative():
    # Eq. dg: d g / dt = C U - B along the motion, with time-dependent links.
    w = small_colony()
    t = 0.13
    S = System(w, t=t)
    rng = np.random.default_rng(1)
    U = rng.standard_normal((S.M_bodies, 6))
    eps = 1e-6
    gs = []
    for sgn in (1, -1):
        q = S.q + sgn * eps * U[:, :3]
        th = quat_mul(quat_from_rotvec(sgn * eps * U[:, 3:]), S.theta)
        dlp, dlq = w["dl"](t + sgn * eps)[:2]
        gs.append(constraint_g(q, th, dlp, dlq, S.bp, S.bq))
    fd = ((gs[0] - gs[1]) / (2 * eps)).ravel()
    CU_B = S.C_dense() @ U.ravel() - S.B_vec()
    assert np.abs(fd - CU_B).max() <= 1e-8 * np.abs(CU_B).max()


def test_A_symmetric(chains_sys):
    A = chains_sys.A_dense()
    assert np.abs(A - A.T).max() == 0.0


def test_dense_and_formal_solutions_agree(chains_sys):
    S = chains_sys
    b = S.rhs()
    yd = S.solve_dense(b)
    yf = S.solve_formal(b)
    A = S.A_dense()
    for y in (yd, yf):
        assert np.linalg.norm(A @ y - b) <= 1e-13 * np.linalg.norm(b)
    assert np.abs(yd - yf).max() <= 1e-12 * np.abs(yd).max()


def test_constraints_and_conservation(chains_sys):
    # C U = B; no net constraint force or torque on an articulated body
    # (App. A); generated power U . C^T phi = phi . B (Sec. 2.2).
    S = chains_sys
    y = S.solve_formal()
    lam, U, phi = S.split(y)
    C = S.C_dense()
    B = S.B_vec()
    assert np.abs(C @ U - B).max() <= 1e-13 * np.abs(U).max()
    FC = (C.T @ phi).reshape(-1, 6)
    for a_ in np.unique(S.assembly):
        bodies = np.nonzero(S.assembly == a_)[0]
        f = FC[bodies, :3].sum(axis=0)
        tau = (FC[bodies, 3:] + np.cross(S.q[bodies], FC[bodies, :3])).sum(axis=0)
        scale = np.abs(FC).max() * (1 + np.abs(S.q).max())
        assert np.abs(f).max() <= 1e-13 * scale
        assert np.abs(tau).max() <= 1e-12 * scale
    assert abs(U @ (C.T @ phi) - phi @ B) <= 1e-12 * np.abs(U).max() * np.abs(phi).max() * len(phi)


def test_projection_is_idempotent(chains_sys):
    # Q = I - N C^T G C with G = (C N C^T)^-1 is a projection (Eq. U).
    S = chains_sys
    K, C, Mm = S.K_dense(), S.C_dense(), S.mobility()
    N = np.linalg.inv(K.T @ np.linalg.solve(Mm, K))
    G = np.linalg.inv(C @ N @ C.T)
    Q = np.eye(len(N)) - N @ C.T @ G @ C
    assert np.abs(Q @ Q - Q).max() <= 1e-10 * np.abs(Q).max()


def test_preconditioner_solves_block_diagonal_problem(chains_sys):
    # P~^-1 r solves Eq. precond (M replaced by its same-body blocks).
    S = chains_sys
    A = S.A_dense()
    nl = 3 * S.Nb
    Mt = np.zeros((nl, nl))
    for p in range(S.M_bodies):
        s = slice(3 * S.off[p], 3 * S.off[p + 1])
        Mt[s, s] = A[s, s]
    At = A.copy()
    At[:nl, :nl] = Mt
    r = np.random.default_rng(4).standard_normal(S.n)
    z = S.apply_preconditioner(r)
    assert np.linalg.norm(At @ z - r) <= 1e-12 * np.linalg.norm(r) * np.abs(At).max()


def test_preconditioner_rank_deficient_pseudo_inverse():
    # Two links between the same pair of rods on their common axis leave
    # C with rank 5 per pair (Sec. 4.3 observes the same for the bacterium
    # hinge); G~ is then a pseudo-inverse and the block-diagonal problem is
    # still solved exactly for consistent right-hand sides.
    w = small_colony()
    S = System(w, t=0.05)
    C = S.C_dense()
    assert np.linalg.matrix_rank(C) == 5 * (len(w["q"]) - 1)
    A = S.A_dense()
    nl = 3 * S.Nb
    for p in range(S.M_bodies):
        s = slice(3 * S.off[p], 3 * S.off[p + 1])
        keep = A[s, s].copy()
        A[:nl, s] = 0.0
        A[s, s] = keep
    # consistent rhs: r3 in range(C)
    rng = np.random.default_rng(8)
    r = rng.standard_normal(S.n)
    nu = 6 * S.M_bodies
    r[nl + nu:] = C @ rng.standard_normal(nu)
    z = S.apply_preconditioner(r)
    assert np.linalg.norm(A @ z - r) <= 1e-10 * np.linalg.norm(r) * np.abs(A).max()


def test_gmres_reaches_dense_solution(chains_sys):
    S = chains_sys
    yd = S.solve_dense()
    yg, its, hist = S.gmres(tol=1e-12)
    assert hist[-1] <= 1e-12
    assert np.abs(yg - yd).max() <= 1e-9 * np.abs(yd).max()


def test_unpreconditioned_gmres_is_slow():
    # Sec. 3.2.1: without preconditioner GMRES needs about as many iterations
    # as unknowns; with it, far fewer.
    w = workloads.chains_free_space(1, n_chains=1, bodies_per_chain=4)
    S = System(w)
    from oracle.system import gmres_right
    b = S.rhs()
    _, it_plain, _ = gmres_right(S.apply_A, lambda v: v, b, tol=1e-8, restart=400, max_iter=400)
    _, it_pc, _ = S.gmres(b=b, tol=1e-8)
    assert it_pc * 2.5 < it_plain
    assert it_plain > 0.3 * S.n


def test_unknown_counts_printed_in_paper():
    # The system sizes the paper prints, from its body/blob/link counts
    # (tests/golden/paper_counts.txt lists them with their sections).
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.txt")
    rows = [l.split("#")[0].split() for l in open(path) if l.strip() and not l.startswith("#")]
    for name, model, blobs, bodies, links, unknowns in rows:
        blobs, bodies, links, unknowns = map(int, (blobs, bodies, links, unknowns))
        if model == "multiblob":
            n = 3 * blobs + 6 * bodies + 3 * links
        else:  # single-blob bodies solve for (phi, U) only (Eq. linear_system_general)
            n = 6 * bodies + 3 * links
        assert n == unknowns, name
