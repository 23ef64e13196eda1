"""Single-blob bodies with rotational coupling on the GPU (through the C ABI)
against the oracle: the body mobility product (generalised RPY tensor,
overlaps included), the constrained solve of Eq. linear_system_general, an
Euler step, two systems in one handle, and the configuration checks."""
import ctypes

import numpy as np
import pytest

from paper_2107_10800_gb300 import build, binding, workloads as W
from oracle import single_blob as osb

pytestmark = pytest.mark.gpu

A = 0.5  # the chains' shells as single blobs: radius 0.5, neighbours 1.05 apart


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.lib()


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def loose(x, a, n_systems=1):
    s = binding.Solver(eta=1.3, a=a, single_blob=True, n_systems=n_systems)
    M = len(x)
    for k in range(n_systems):
        s.set_bodies(x, np.tile([1.0, 0, 0, 0], (M, 1)), None, None, np.zeros((M, 6)), np.arange(M), system=k)
    return s


@pytest.mark.parametrize("M", [1, 7, 130, 300])
def test_body_mobility_matches_oracle(M):
    rng = np.random.default_rng(M)
    x = rng.uniform(0.0, max(1.0, (M / 4.0) ** (1 / 3)), (M, 3))  # dense: many overlaps at a = 0.3
    g = rng.standard_normal((M, 6))
    s = loose(x, 0.3)
    ref = (osb.grand_mobility(x, 0.3, 1.3) @ g.ravel()).reshape(-1, 6)
    assert rel(s.apply_mobility(g), ref) <= 1e-12


def test_body_mobility_two_systems():
    rng = np.random.default_rng(5)
    x = rng.uniform(0.0, 3.0, (150, 3))
    g = rng.standard_normal((300, 6))
    s = loose(x, 0.3, n_systems=2)
    N = osb.grand_mobility(x, 0.3, 1.3)
    u = s.apply_mobility(g)
    assert rel(u[:150], (N @ g[:150].ravel()).reshape(-1, 6)) <= 1e-12
    assert rel(u[150:], (N @ g[150:].ravel()).reshape(-1, 6)) <= 1e-12


def test_constrained_solve_matches_oracle():
    w = dict(W.chains_free_space(7, n_chains=3, bodies_per_chain=6), a=A)
    o = osb.SingleBlobSystem(w)
    U_o, phi_o = o.solve_dense()
    s = binding.Solver.from_workload(w, tol=1e-13, single_blob=True)
    U, phi, lam, st = s.solve()
    assert st["status"] == 0 and st["rel_residual"] <= 1e-13
    assert lam.size == 0
    assert rel(U.ravel(), U_o) <= 1e-10
    C = o.S.C_dense()
    assert rel(C.T @ phi.ravel(), C.T @ phi_o) <= 1e-9
    assert np.abs(C @ U.ravel() - o.S.B_vec()).max() <= 1e-12 * np.abs(U).max()


def test_euler_step_matches_oracle():
    w = dict(W.chains_free_space(8, n_chains=2, bodies_per_chain=5), a=A)
    o = osb.SingleBlobSystem(w)
    dl0 = (o.S.dl_p, o.S.dl_q, None, None)
    dt = 5e-2
    s = binding.Solver.from_workload(w, tol=1e-13, single_blob=True)
    s.step(0.0, dt)
    q, th = s.bodies()
    qo, tho, _ = osb.euler_step(w, w["q"], w["theta"], 0.0, dt, dl_now=dl0)
    assert rel(q, qo) <= 1e-10
    assert rel(th, tho) <= 1e-10


def test_single_blob_configuration_checks():
    L = binding.lib()
    for wall, prec, sbv in ((1, 0, 1), (0, 1, 1), (0, 0, 2)):
        cfg = binding.Config(1.0, 0.1, wall, prec, 1, 1e-8, 50, 100, 1e-10, 10, None, sbv)
        h = ctypes.c_void_p()
        assert L.am_create(ctypes.byref(cfg), ctypes.byref(h)) == binding.AM_ERR_ARG
