"""The seeded workloads have the sizes and structure stated for them, and
start with satisfied constraints (checked with the oracle)."""
import numpy as np
import pytest

from paper_2107_10800_gb300 import workloads as W
from oracle.system import System
from oracle.timestep import constraint_g


def test_chains_sizes_and_joints():
    w = W.chains_free_space(1)
    assert W.counts(w) == (384, 32, 28, 1428)
    S = System(w)
    assert np.abs(constraint_g(S.q, S.theta, S.dl_p, S.dl_q, S.bp, S.bq)).max() < 1e-14
    assert np.allclose(np.linalg.norm(w["theta"], axis=1), 1.0, atol=1e-15)
    steps = np.linalg.norm(np.diff(w["q"].reshape(4, 8, 3), axis=1), axis=2)
    assert np.allclose(steps, 1.05)
    assert np.all(w["q"] >= 0) and np.all(w["q"] <= 10)


def test_colony_sizes_and_sliding_links():
    w = W.diatom_colony(1)
    assert W.counts(w) == (2560, 32, 62, 8058)
    for t in (0.0, 0.037):
        S = System(w, t=t)
        g = constraint_g(S.q, S.theta, S.dl_p, S.dl_q, S.bp, S.bq)
        if t == 0.0:
            assert np.abs(g).max() < 1e-15
    assert S.r[:, 2].min() > w["a"]
    # dL/dt is the derivative of L
    eps = 1e-6
    dp1 = (w["dl"](0.3 + eps)[0] - w["dl"](0.3 - eps)[0]) / (2 * eps)
    assert np.allclose(dp1, w["dl"](0.3)[2], atol=1e-8)


def test_bacteria_sizes_and_joints():
    w = W.bacteria_wall(4, n_bact=3)
    nb, M, P, n = W.counts(w)
    assert (nb, M, P) == (3 * 360, 3 * 17, 3 * 17)
    S = System(w)
    assert np.abs(constraint_g(S.q, S.theta, S.dl_p, S.dl_q, S.bp, S.bq)).max() < 1e-13
    assert S.r[:, 2].min() > w["a"]
    # the hinge (first two links of a bacterium) has rank 5 of 6
    C = S.C_dense()
    hinge = C[0:6, 0:12]
    assert np.linalg.matrix_rank(hinge) == 5
    # the full-size workload: 1,000 bacteria, 360,000 blobs
    full = 1000 * 360
    assert full == 360_000


def test_seeds_are_reproducible():
    a = W.chains_free_space(5)
    b = W.chains_free_space(5)
    assert np.array_equal(a["q"], b["q"]) and np.array_equal(a["F"], b["F"])
    c = W.chains_free_space(6)
    assert not np.array_equal(a["q"], c["q"])


def test_batched_chains_sizes():
    ws = W.batched_chains(1)
    nb = np.array([W.counts(w)[0] for w in ws])
    assert len(ws) == 256
    assert nb.min() >= 500 - 12 and nb.max() <= 20_000 + 12
    assert np.all(nb % 12 == 0)
    # log-uniform: the median is near the geometric mean of the bounds
    assert 2000 < np.median(nb) < 5000
    for w in ws[:5]:
        S = System(w)
        assert np.abs(constraint_g(S.q, S.theta, S.dl_p, S.dl_q, S.bp, S.bq)).max() < 1e-13
