"""What a low-rank correction of the block-diagonal preconditioner can gain
at best (the learned form's second output; Sec. 3.1 for the preconditioner
being corrected).  CPU, oracle only.

For each articulated body a (here: a bacterium of 17 bodies, 360 blobs,
1,233 unknowns) the correction that would turn the block-diagonal
preconditioner P~ into the exact solve of a's own saddle-point problem is
D_a = (A_aa)^+ - P~_aa^-1.  Its best rank-k approximation (truncated SVD) is
the most any rank-k correction of a's block can add, learned or not.  The
test runs right-preconditioned GMRES (the oracle's) to 1e-8 on two bacteria
above a wall at the density of the 1,000-bacteria suspension with:
  - P~ alone,
  - P~ plus the best rank-8 correction per articulated body,
  - P~ with the (U, phi) rows corrected exactly and lambda recomputed from
    the block-diagonal M~ as P~ does (the correction in body-velocity
    space that a per-body 6 x 8 output could express, at its ceiling),
  - the exact per-articulated-body solve.
Measured here: 16, 16, 20 and 3 iterations: the blob-level hydrodynamics
between the bodies of one bacterium carry the gain, and D_a has no
low-rank part (its singular values fall slowly), so a rank-8 correction
gains nothing."""
import numpy as np

from oracle.system import System, gmres_right
from paper_2107_10800_gb300 import learned


def test_rank8_correction_ceiling():
    w = learned.bacteria_at_density(20000, 2)
    S = System(w)
    A = S.A_dense()
    S.build_preconditioner()
    b = S.rhs()
    n, nl, nu = S.n, 3 * S.Nb, 6 * S.M_bodies
    asm = np.asarray(S.assembly)
    sets = []
    for a_ in np.unique(asm):
        bodies = np.nonzero(asm == a_)[0]
        lam = np.concatenate([np.arange(3 * S.off[p], 3 * S.off[p + 1]) for p in bodies])
        U = np.concatenate([nl + np.arange(6 * p, 6 * p + 6) for p in bodies])
        links = np.nonzero(asm[S.bp] == a_)[0]
        phi = np.concatenate([nl + nu + np.arange(3 * q, 3 * q + 3) for q in links])
        sets.append(np.concatenate([lam, U, phi]))
    exact = [np.linalg.pinv(A[np.ix_(I, I)], rcond=1e-12) for I in sets]
    blocks = []  # P~ restricted to each articulated body, column by column
    for I in sets:
        E = np.zeros((len(I), len(I)))
        for c in range(len(I)):
            e = np.zeros(n)
            e[I[c]] = 1.0
            E[:, c] = S.apply_preconditioner(e)[I]
        blocks.append(E)

    def iterations(P):
        return gmres_right(lambda y: A @ y, P, b, tol=1e-8, restart=50, max_iter=500)[1]

    it_block = iterations(S.apply_preconditioner)

    def P_exact(r):
        y = np.zeros_like(r)
        for I, X in zip(sets, exact):
            y[I] = X @ r[I]
        return y

    it_exact = iterations(P_exact)

    best8 = []
    for I, X, E in zip(sets, exact, blocks):
        Uu, s, Vt = np.linalg.svd(X - E)
        best8.append((I, Uu[:, :8] * s[:8], Vt[:8]))
        assert s[8] > 0.5 * s[0]  # no low-rank part: the ninth value is still large

    def P_rank8(r):
        y = S.apply_preconditioner(r)
        for I, Us, Vt in best8:
            y[I] += Us @ (Vt @ r[I])
        return y

    it_rank8 = iterations(P_rank8)

    Minv, K = S._pc_Minv, S._pc_K

    def P_velocity(r):
        y = S.apply_preconditioner(r)
        for I, X in zip(sets, exact):
            sel = I >= nl
            y[I[sel]] = (X @ r[I])[sel]
        t = r[:nl] + K @ y[nl:nl + nu]
        for p in range(S.M_bodies):
            s_ = slice(3 * S.off[p], 3 * S.off[p + 1])
            y[s_] = Minv[p] @ t[s_]
        return y

    it_velocity = iterations(P_velocity)
    assert it_block >= 12
    assert it_rank8 >= it_block - 1, (it_block, it_rank8)
    assert it_velocity >= it_block - 1, (it_block, it_velocity)
    assert it_exact <= it_block // 2, (it_block, it_exact)


def test_global_rank8_deflation_ceiling():
    # The other form a rank-8 term can take: a global coarse correction.  Its
    # ceiling moves the 8 eigenvalues of A P~^-1 nearest zero (the null
    # directions of the redundant links left out) to 1 exactly: with right
    # eigenvectors V and left ones W (W^T V = I), P^-1 = P~^-1 (I + V
    # (L^-1 - I) W^T).  On two bacteria the spectrum has a cluster of 15
    # eigenvalues per bacterium near 0.36, so deflating 8 gains nothing
    # (measured here 16 -> 16; 4 bacteria 16 -> 17; the 32-body diatom
    # colony 39 -> 38, rank 32: 35).
    w = learned.bacteria_at_density(20000, 2)
    S = System(w)
    A = S.A_dense()
    S.build_preconditioner()
    b = S.rhs()
    n = S.n
    Pinv = np.column_stack([S.apply_preconditioner(e) for e in np.eye(n)])
    lam, V = np.linalg.eig(A @ Pinv)
    Wt = np.linalg.inv(V)
    order = np.argsort(np.abs(lam))
    order = order[np.abs(lam[order]) > 1e-8]
    assert np.sum(np.abs(lam[order]) < 0.4) >= 15 * 2  # the cluster
    sel = set(order[:8].tolist())
    for i in list(sel):  # conjugate partners keep the correction real
        if abs(lam[i].imag) > 0:
            sel.add(int(np.argmin(np.abs(lam - np.conj(lam[i])))))
    idx = np.array(sorted(sel))
    corr = ((V[:, idx] * (1.0 / lam[idx] - 1.0)) @ Wt[idx, :]).real

    def iterations(P):
        return gmres_right(lambda y: A @ y, P, b, tol=1e-8, restart=50, max_iter=500)[1]

    it_plain = iterations(S.apply_preconditioner)
    it_defl = iterations(lambda r: Pinv @ (r + corr @ r))
    assert it_plain >= 12
    assert it_defl >= it_plain - 1, (it_plain, it_defl)
