"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: FP64 path within 1e-10 relative of the oracle (the mobility product
and operator within 1e-12); mixed path within 1e-5.  Relative errors are
max-abs differences over the max-abs of the oracle value."""
import numpy as np
import pytest

from paper_2107_10800_gb300 import build, binding, workloads as W
from oracle import mobility as om
from oracle.system import System
from oracle import timestep as ots

pytestmark = pytest.mark.gpu

FP64_MATVEC = 1e-12
FP64_SOLVE = 1e-10
MIXED = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.lib()


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def loose_blobs_solver(r, a, wall, precision):
    """A solver whose bodies are single blobs (only for mobility products)."""
    n = len(r)
    s = binding.Solver(eta=1.0, a=a, wall=wall, precision=precision)
    theta = np.tile([1.0, 0, 0, 0], (n, 1))
    s.set_bodies(r, theta, np.arange(n + 1), np.zeros((n, 3)), np.zeros((n, 6)), np.arange(n))
    return s


@pytest.mark.parametrize("n", [1, 2, 13, 129, 300, 1000])
@pytest.mark.parametrize("wall", [0, 1])
def test_mobility_fp64_matches_oracle(n, wall):
    r, lam = W.random_blobs(100 + n, n, a=0.1, wall=wall)
    s = loose_blobs_solver(r, 0.1, wall, "fp64")
    u = s.apply_mobility(lam)
    ref = om.mobility_matvec(r, lam, 0.1, 1.0, wall)
    assert rel(u, ref) <= FP64_MATVEC


@pytest.mark.parametrize("n", [13, 1000])
@pytest.mark.parametrize("wall", [0, 1])
def test_mobility_mixed_matches_oracle(n, wall):
    r, lam = W.random_blobs(200 + n, n, a=0.1, wall=wall)
    r = r + np.array([250.0, -125.0, 0.0])  # far from the origin: hi/lo positions matter
    s = loose_blobs_solver(r, 0.1, wall, "mixed")
    u = s.apply_mobility(lam)
    ref = om.mobility_matvec(r, lam, 0.1, 1.0, wall)
    assert rel(u, ref) <= MIXED


DF64_MATVEC = 1e-11


@pytest.mark.parametrize("n", [13, 300, 1000])
@pytest.mark.parametrize("wall", [0, 1])
def test_mobility_df64_matches_oracle(n, wall):
    # double-float pair terms (the mixed solver's outer residual), positions
    # far from the origin so that the hi/lo split of the positions matters
    r, lam = W.random_blobs(300 + n, n, a=0.1, wall=wall)
    r = r + np.array([250.0, -125.0, 0.0])
    for prec in ("mixed", "fp64"):
        s = loose_blobs_solver(r, 0.1, wall, prec)
        ref = om.mobility_matvec(r, lam, 0.1, 1.0, wall)
        assert rel(s.apply_mobility_ex(lam, "df64"), ref) <= DF64_MATVEC
        assert rel(s.apply_mobility_ex(lam, "fp64"), ref) <= FP64_MATVEC
        assert rel(s.apply_mobility_ex(lam, "mixed"), ref) <= MIXED


def test_mobility_df64_overlap_and_contact():
    r = np.array([[0, 0, 1.0], [0.05, 0, 1.0], [0.25, 0, 1.0], [0.25, 0.2, 1.0], [0.25, 0.2, 1.0],
                  [0.45, 0.2, 1.0]])
    lam = np.random.default_rng(1).standard_normal(r.shape)
    for wall in (0, 1):
        s = loose_blobs_solver(r, 0.1, wall, "mixed")
        ref = om.mobility_matvec(r, lam, 0.1, 1.0, wall)
        assert rel(s.apply_mobility_ex(lam, "df64"), ref) <= DF64_MATVEC


@pytest.mark.parametrize("wall", [0, 1])
@pytest.mark.parametrize("layout", [(1, 0), (2, 0), (2, 96), (1, 300), (2, 300)])
def test_mobility_mixed_layouts_match_oracle(wall, layout):
    # every work-item layout of the mixed product, including two targets per
    # thread in paired FP32 lanes, ragged items and overlapping blobs
    r, lam = W.random_blobs(400 + wall, 1000, a=0.1, wall=wall)
    r = r + np.array([250.0, -125.0, 0.0])
    r[1] = r[0] + np.array([0.05, 0.0, 0.0])      # overlapping pair
    r[200] = r[1] + np.array([0.0, 0.2, 0.0])     # contact at 2a
    s = loose_blobs_solver(r, 0.1, wall, "mixed")
    s.set_mobility_layout(*layout)
    ref = om.mobility_matvec(r, lam, 0.1, 1.0, wall)
    for _ in range(2):
        assert rel(s.apply_mobility_ex(lam, "mixed"), ref) <= MIXED
    assert rel(s.apply_mobility_ex(lam, "df64"), ref) <= DF64_MATVEC


def test_solve_mixed_with_paired_layout_matches_oracle():
    w = small_colony(4)
    S = System(w, t=0.02)
    s = binding.Solver.from_workload(w, t=0.02, tol=1e-9, precision="mixed")
    s.set_mobility_layout(2, 64)
    U, phi, lam, st = s.solve()
    assert st["status"] == 0 and st["rel_residual"] <= 1e-9
    lam_o, U_o, _ = S.split(S.solve_formal())
    assert rel(U.ravel(), U_o) <= MIXED


def test_mobility_overlap_and_contact():
    # overlapping blobs (r < 2a), exact contact (r = 2a) and coincident
    # free-space blobs (r = 0 between distinct blobs gives mu0 I)
    r = np.array([[0, 0, 1.0], [0.05, 0, 1.0], [0.25, 0, 1.0], [0.25, 0.2, 1.0], [0.25, 0.2, 1.0]])
    lam = np.random.default_rng(0).standard_normal(r.shape)
    for wall in (0, 1):
        s = loose_blobs_solver(r, 0.1, wall, "fp64")
        assert rel(s.apply_mobility(lam), om.mobility_matvec(r, lam, 0.1, 1.0, wall)) <= FP64_MATVEC


def test_stateless_matvec_matches_oracle():
    torch = pytest.importorskip("torch")
    n = 777
    r, lam = W.random_blobs(5, n, a=0.1, wall=1)
    ref = om.mobility_matvec(r, lam, 0.1, 1.0, 1)
    dev = torch.device("cuda")
    for prec, bar in (("fp64", FP64_MATVEC), ("mixed", MIXED)):
        dr = torch.tensor(r, device=dev)
        dl = torch.tensor(lam, device=dev)
        du = torch.empty_like(dr)
        nbytes = binding.rpy_matvec_workspace(n, prec)
        work = torch.empty(nbytes // 8 + 64, dtype=torch.float64, device=dev)
        base = work.data_ptr()
        aligned = (base + 255) // 256 * 256
        binding.rpy_matvec_ptr(dr.data_ptr(), dl.data_ptr(), du.data_ptr(), n, 1.0, 0.1, 1, prec,
                               aligned, nbytes, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert rel(du.cpu().numpy(), ref) <= bar


@pytest.fixture(scope="module")
def chains():
    w = W.chains_free_space(1)
    return w, System(w)


def test_pose_matches_oracle(chains):
    w, S = chains
    s = binding.Solver.from_workload(w)
    assert rel(s.blobs(), S.r) <= 1e-15


def test_operator_matches_oracle(chains):
    w, S = chains
    s = binding.Solver.from_workload(w)
    y = np.random.default_rng(1).standard_normal(S.n)
    assert rel(s.apply_operator(y), S.apply_A(y)) <= FP64_MATVEC


def test_preconditioner_matches_oracle(chains):
    w, S = chains
    s = binding.Solver.from_workload(w)
    r = np.random.default_rng(2).standard_normal(S.n)
    assert rel(s.apply_precond(r), S.apply_preconditioner(r)) <= FP64_SOLVE


def test_preconditioner_fp32_storage_matches_oracle(chains):
    # mixed handles keep the preconditioner's matrices in FP32
    w, S = chains
    s = binding.Solver.from_workload(w, precision="mixed")
    r = np.random.default_rng(3).standard_normal(S.n)
    assert rel(s.apply_precond(r), S.apply_preconditioner(r)) <= 1e-4


def test_preconditioner_cluster_build_matches_oracle():
    # 12 rods of 2 x 40 blobs (240 rows each) and one articulated body of 22
    # links (66 rows, rank 55): both builds take clusters of CTAs.  The link
    # block of r lies in range(C), where every generalised inverse of
    # C N~ C^T gives the same lambda, U and C^T phi.  FP32 storage: the
    # error is bounded by about kappa * 2^-24 with kappa = 1.1e4 for
    # C N~ C^T on range(C) here (M^(pp): 43), i.e. 6.6e-4; bar 2e-3.
    w = W.diatom_colony(5, n_rods=12, nx=40)
    S = System(w)
    rng = np.random.default_rng(4)
    r = rng.standard_normal(S.n)
    C = S.C_dense()
    nl, nu = 3 * S.Nb, 6 * S.M_bodies
    r[nl + nu:] = C @ rng.standard_normal(nu)
    lam_o, U_o, phi_o = S.split(S.apply_preconditioner(r))
    for precision, bar in (("fp64", FP64_SOLVE), ("mixed", 2e-3)):
        s = binding.Solver.from_workload(w, precision=precision)
        lam, U, phi = S.split(s.apply_precond(r))
        assert rel(lam, lam_o) <= bar
        assert rel(U, U_o) <= bar
        assert rel(C.T @ phi, C.T @ phi_o) <= bar


def test_solve_chains_matches_dense_solution(chains):
    w, S = chains
    s = binding.Solver.from_workload(w, tol=1e-13)
    U, phi, lam, st = s.solve()
    y = S.solve_dense()
    lam_o, U_o, phi_o = S.split(y)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-13
    assert rel(U.ravel(), U_o) <= FP64_SOLVE
    assert rel(lam.ravel(), lam_o) <= FP64_SOLVE
    assert rel(phi.ravel(), phi_o) <= FP64_SOLVE
    assert st["constraint_residual"] <= 1e-13 * np.abs(U).max()


def small_colony(seed=3, n_rods=8, nx=10):
    return W.diatom_colony(seed, n_rods=n_rods, nx=nx)


def test_solve_colony_rank_deficient_matches_oracle():
    # wall + two links per rod pair (rank-deficient C): lambda, U and C^T phi
    # are unique; phi is compared through C^T phi.
    w = small_colony()
    t = 0.07
    S = System(w, t=t)
    s = binding.Solver.from_workload(w, t=t, tol=1e-13)
    U, phi, lam, st = s.solve()
    y = S.solve_formal()
    lam_o, U_o, phi_o = S.split(y)
    C = S.C_dense()
    assert st["status"] == 0
    assert rel(U.ravel(), U_o) <= FP64_SOLVE
    assert rel(lam.ravel(), lam_o) <= FP64_SOLVE
    assert rel(C.T @ phi.ravel(), C.T @ phi_o) <= FP64_SOLVE
    assert st["constraint_residual"] <= 1e-12 * np.abs(U).max()


def test_solve_mixed_reaches_fp64_residual():
    w = small_colony(4)
    S = System(w, t=0.02)
    s = binding.Solver.from_workload(w, t=0.02, tol=1e-8, precision="mixed")
    U, phi, lam, st = s.solve()
    assert st["status"] == 0 and st["rel_residual"] <= 1e-8
    y = S.solve_formal()
    lam_o, U_o, _ = S.split(y)
    assert rel(U.ravel(), U_o) <= MIXED
    assert rel(lam.ravel(), lam_o) <= MIXED


def test_solve_mixed_tight_tolerance_true_residual():
    # The refinement stops on a double-float residual, or on the inner
    # solve's mixed residual plus a bound on the mixed product's error (after
    # a correction computed from a double-float residual).  Either way the
    # reported residual bounds the true one: the oracle's FP64 residual of the
    # returned solution is below it (up to the double-float residual's own
    # rounding) and within the tolerance.
    w = small_colony(5)
    S = System(w, t=0.03)
    s = binding.Solver.from_workload(w, t=0.03, tol=1e-11, precision="mixed")
    U, phi, lam, st = s.solve()
    assert st["status"] == 0 and st["rel_residual"] <= 1e-11
    y = np.concatenate([lam.ravel(), U.ravel(), phi.ravel()])
    b = S.rhs()
    true_rel = np.linalg.norm(b - S.apply_A(y)) / np.linalg.norm(b)
    assert true_rel <= st["rel_residual"] + 1e-12, (true_rel, st["rel_residual"])


def test_euler_step_open_chains_matches_oracle(chains):
    w, S = chains
    dt = 1e-2
    s = binding.Solver.from_workload(w, tol=1e-13)
    U, phi, lam, st = s.step(0.0, dt)
    q, th = s.bodies()
    qo, tho, info = ots.euler_step(w, w["q"], w["theta"], 0.0, dt, delta=1e-10, solve_tol=1e-13)
    assert st["status"] == 0
    assert rel(q, qo) <= FP64_SOLVE
    assert rel(th, tho) <= FP64_SOLVE
    assert st["corr_iterations"] == 0 and st["g2_before"] < 1e-24


def test_euler_step_colony_with_correction_matches_oracle():
    w = small_colony(5, n_rods=6, nx=8)
    t, dt = 0.1, 2e-2
    s = binding.Solver.from_workload(w, t=t, tol=1e-13)
    dlp1, dlq1 = w["dl"](t + dt)[:2]
    U, phi, lam, st = s.step(t, dt, dl_next=(dlp1, dlq1))
    q, th = s.bodies()
    qo, tho, info = ots.euler_step(w, w["q"], w["theta"], t, dt, delta=1e-10, solve_tol=1e-13)
    assert info["g2_before"] >= 1e-10  # the correction ran on both sides
    assert st["g2_before"] == pytest.approx(info["g2_before"], rel=1e-6)
    assert st["corr_iterations"] >= 1 and st["g2_after"] < 1e-20
    assert rel(q, qo) <= FP64_SOLVE
    assert rel(th, tho) <= FP64_SOLVE


def test_wall_penetration_is_an_error():
    w = small_colony(6, n_rods=2, nx=4)
    w = dict(w)
    w["q"] = w["q"].copy()
    w["q"][0, 2] = 0.05  # below a = 0.1
    s = binding.Solver(eta=1.0, a=0.1, wall=1)
    with pytest.raises(binding.AmError) as e:
        s.set_bodies(w["q"], w["theta"], w["blob_offset"], w["rho"], w["F"], w["assembly"])
    assert e.value.code == binding.AM_ERR_WALL_PENETRATION


def test_bad_inputs_are_errors(chains):
    w, S = chains
    s = binding.Solver(eta=1.0, a=0.1, wall=0)
    th = w["theta"].copy()
    th[3] *= 1.5
    with pytest.raises(binding.AmError) as e:
        s.set_bodies(w["q"], th, w["blob_offset"], w["rho"], w["F"], w["assembly"])
    assert e.value.code == binding.AM_ERR_NONUNIT_QUAT
    s.set_bodies(w["q"], w["theta"], w["blob_offset"], w["rho"], w["F"], w["assembly"])
    with pytest.raises(binding.AmError):
        s.set_constraints([0], [0], np.zeros(3), np.zeros(3))      # body linked to itself
    with pytest.raises(binding.AmError):
        s.set_constraints([0], [9], np.zeros(3), np.zeros(3))      # across articulated bodies
    # single-blob bodies have a singular body mobility without rotational RPY
    r, _ = W.random_blobs(1, 10)
    s2 = loose_blobs_solver(r, 0.1, 0, "fp64")
    with pytest.raises(binding.AmError) as e:
        s2.solve()
    assert e.value.code == binding.AM_ERR_SINGULAR


def test_not_converged_reports_status(chains):
    w, S = chains
    s = binding.Solver.from_workload(w, tol=1e-14, max_iter=3)
    U, phi, lam, st = s.solve()
    assert st["status"] == binding.AM_ERR_NOT_CONVERGED
    assert st["iterations"] == 3
    assert np.all(np.isfinite(U))


# --------------------------------------------------------- full sizes ---
@pytest.mark.slow
def test_colony_full_size_solve():
    # 2,560 blobs, wall, 62 links (8,058 unknowns, C of rank 155): a solve
    # to relative residual 1e-12 agrees with the oracle's dense solve of the
    # whole saddle-point system at the FP64 bar, in lambda, U and C^T phi
    # (phi itself is unique only modulo null(C^T)); sampled mobility rows
    # agree with the oracle's rows.  The errors follow the residual (the
    # oracle's dense and formal solutions agree to about 5e-13).
    w = W.diatom_colony(1)
    t = 0.05
    S = System(w, t=t)
    s = binding.Solver.from_workload(w, t=t, tol=1e-12, max_iter=2000)
    rows = np.random.default_rng(0).choice(S.Nb, 64, replace=False)
    lam = np.random.default_rng(1).standard_normal((S.Nb, 3))
    u = s.apply_mobility(lam)
    assert rel(u[rows], om.mobility_rows(S.r, lam, rows, S.a, S.eta, 1)) <= FP64_MATVEC
    U, phi, lamg, st = s.solve()
    assert st["status"] == 0 and st["rel_residual"] <= 1e-12
    lam_o, U_o, phi_o = S.split(S.solve_dense())
    C = S.C_dense()
    assert rel(lamg.ravel(), lam_o) <= FP64_SOLVE
    assert rel(U.ravel(), U_o) <= FP64_SOLVE
    assert rel(C.T @ phi.ravel(), C.T @ phi_o) <= FP64_SOLVE


@pytest.mark.slow
def test_bacteria_full_size_mobility_sampled():
    # 360,000 blobs above a wall: the mixed product on sampled target rows;
    # the FP64 product on a 40,000-blob subset (same geometry).
    w = W.bacteria_wall(1)
    s = binding.Solver.from_workload(w, precision="mixed")
    r = s.blobs()
    assert r.shape == (360_000, 3) and r[:, 2].min() > w["a"]
    lam = np.random.default_rng(2).standard_normal(r.shape)
    u = s.apply_mobility(lam)
    rows = np.random.default_rng(3).choice(len(r), 6, replace=False)
    ref = om.mobility_rows(r, lam, rows, w["a"], w["eta"], 1)
    assert rel(u[rows], ref) <= MIXED
    sub = slice(0, 40_000)
    s64 = loose_blobs_solver(r[sub], w["a"], 1, "fp64")
    u64 = s64.apply_mobility(lam[sub])
    rows = np.random.default_rng(4).choice(40_000, 16, replace=False)
    ref = om.mobility_rows(r[sub], lam[sub], rows, w["a"], w["eta"], 1)
    assert rel(u64[rows], ref) <= FP64_MATVEC
