"""Learned warm start: per-body features and the MLP (TEST INFRASTRUCTURE
ONLY: CPU oracle, FP64).

The paper has no learned component; this module is the oracle of the
library's learned warm start.  Its kernels must reproduce:

Features of body p, in the body frame of p (FEAT = 128 values):
  for the K = 16 nearest other bodies k of the same system (by |q_k - q_p|
  rounded to 1e-8, then by body index; zeros when there are fewer):
      R_p^T (q_k - q_p) / L            3 values
      theta_p^* . theta_k, sign s >= 0  4 values  (relative orientation)
  then  q_p,z / L                       height (0 in free space)
        R_p^T f_p, R_p^T tau_p          6 values
        R_p^T u_pc, R_p^T omega_pc      6 values: body velocity of the
                                        block-diagonal solution P~^-1 b
        log(blobs of p) / 5             1 value
  and zeros up to 128; L = 4.
Target: the background flow of the body.  The solution satisfies
M lambda - K U = u_s; its block-diagonal part M~ lambda (blobs of the same
body only) is what the body's own forces do, so u_ext = (M - M~) lambda is
the flow the other bodies induce at its blobs.  Its target is the body-frame
fit of u_ext by NFLOW = 29 flows on the body-frame blob offsets rho
(translation 3, rotation 3, traceless symmetric strain 5, quadratic 18, see
flow_basis): the coefficients c_p minimising |B_p c - R_p^T u_ext,p|^2 +
eps |c|^2 with eps = RIDGE tr(B_p^T B_p) / NFLOW, zero padded to OUT = 32.
The initial guess solves the block-diagonal problem with the predicted flow
moved to the right-hand side: x0 = P~^-1 (u_s - u_fit, -F, B), u_fit at
blob i of body p = R_p B_p(rho_i) c_p.

MLP (DEPTH = 3 hidden layers of WIDTH = 256, ReLU):
  a0 = (x - mu) / sd;  a_l = relu(a_{l-1} W_l^T + b_l), l = 1..3;
  y_n = a3 W4^T + b4;  prediction y = y_n * sd_out.
Loss (training): mean over samples and the OUT outputs of
  (y_n - t / sd_out)^2.
Parameters are flattened in the order W1, b1, W2, b2, W3, b3, W4, b4
(W_l row-major, out x in).
"""
import numpy as np

from .kinematics import rotation_matrix, quat_mul

FEAT = 128
OUT = 32
NFLOW = 29
RIDGE = 1e-6
WIDTH = 256
DEPTH = 3
KNN = 16
LSCALE = 4.0


def features(q, theta, F, blob_offset, U_pc, system_of_body, wall):
    """(M, FEAT) features of every body (see module docstring)."""
    q = np.asarray(q, float)
    theta = np.asarray(theta, float)
    F = np.asarray(F, float).reshape(-1, 6)
    U_pc = np.asarray(U_pc, float).reshape(-1, 6)
    M = len(q)
    R = rotation_matrix(theta)
    X = np.zeros((M, FEAT))
    conj = theta * np.array([1.0, -1.0, -1.0, -1.0])
    nblob = np.diff(np.asarray(blob_offset))
    sysb = np.asarray(system_of_body)
    for p in range(M):
        same = np.nonzero(sysb == sysb[p])[0]
        same = same[same != p]
        d = np.linalg.norm(q[same] - q[p], axis=1)
        key = np.floor(d * 1e8 + 0.5)  # ties (equal distances) broken by body index
        order = same[np.lexsort((same, key))][:KNN]
        for slot, k in enumerate(order):
            X[p, 7 * slot:7 * slot + 3] = R[p].T @ (q[k] - q[p]) / LSCALE
            rq = quat_mul(conj[p], theta[k])
            if rq[0] < 0:
                rq = -rq
            X[p, 7 * slot + 3:7 * slot + 7] = rq
        base = 7 * KNN
        X[p, base] = q[p, 2] / LSCALE if wall else 0.0
        X[p, base + 1:base + 4] = R[p].T @ F[p, :3]
        X[p, base + 4:base + 7] = R[p].T @ F[p, 3:]
        X[p, base + 7:base + 10] = R[p].T @ U_pc[p, :3]
        X[p, base + 10:base + 13] = R[p].T @ U_pc[p, 3:]
        X[p, base + 13] = np.log(nblob[p]) / 5.0
    return X


# monomials of the quadratic flows, in column order
_QUAD = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def flow_basis(rho):
    """(3n, NFLOW) body-frame flows at the offsets rho (n, 3); row 3i + c is
    velocity component c at blob i.  Columns: e_k (k = 0..2); e_k x rho
    (k = 0..2); E rho for the strains E01, E02, E12 (symmetric unit
    off-diagonal pairs), diag(1, -1, 0), diag(1, 0, -1); then for each
    component c and monomial (i, j) in _QUAD the flow rho_i rho_j e_c."""
    rho = np.asarray(rho, float)
    n = len(rho)
    B = np.zeros((n, 3, NFLOW))
    for k in range(3):
        B[:, k, k] = 1.0
        e = np.zeros(3)
        e[k] = 1.0
        B[:, :, 3 + k] = np.cross(e, rho)
    strains = []
    for (i, j) in ((0, 1), (0, 2), (1, 2)):
        E = np.zeros((3, 3))
        E[i, j] = E[j, i] = 1.0
        strains.append(E)
    strains.append(np.diag([1.0, -1.0, 0.0]))
    strains.append(np.diag([1.0, 0.0, -1.0]))
    for k, E in enumerate(strains):
        B[:, :, 6 + k] = rho @ E.T
    for c in range(3):
        for m, (i, j) in enumerate(_QUAD):
            B[:, c, 11 + 6 * c + m] = rho[:, i] * rho[:, j]
    return B.reshape(3 * n, NFLOW)


def background_flow(M_dense, lam, blob_offset):
    """u_ext = (M - M~) lambda: the full mobility product minus the blocks of
    blobs of the same body."""
    lam = np.asarray(lam, float).ravel()
    u = M_dense @ lam
    off = np.asarray(blob_offset)
    for p in range(len(off) - 1):
        s = slice(3 * off[p], 3 * off[p + 1])
        u[s] -= M_dense[s, s] @ lam[s]
    return u


def flow_targets(theta, rho, blob_offset, u_ext, ridge=RIDGE):
    """(M, OUT) ridge fits of the body-frame background flow (module
    docstring), zero padded."""
    R = rotation_matrix(np.asarray(theta, float))
    off = np.asarray(blob_offset)
    u = np.asarray(u_ext, float).reshape(-1, 3)
    T = np.zeros((len(off) - 1, OUT))
    for p in range(len(off) - 1):
        B = flow_basis(np.asarray(rho)[off[p]:off[p + 1]])
        ub = (u[off[p]:off[p + 1]] @ R[p]).ravel()  # rows R_p^T u_i
        G = B.T @ B
        eps = ridge * np.trace(G) / NFLOW
        T[p, :NFLOW] = np.linalg.solve(G + eps * np.eye(NFLOW), B.T @ ub)
    return T


def flow_field(theta, rho, blob_offset, C):
    """(Nb, 3) lab-frame flow u_fit of the coefficients C (M, >= NFLOW)."""
    R = rotation_matrix(np.asarray(theta, float))
    off = np.asarray(blob_offset)
    out = np.zeros((off[-1], 3))
    for p in range(len(off) - 1):
        B = flow_basis(np.asarray(rho)[off[p]:off[p + 1]])
        out[off[p]:off[p + 1]] = (B @ np.asarray(C, float)[p, :NFLOW]).reshape(-1, 3) @ R[p].T
    return out


def shapes():
    dims = [FEAT] + [WIDTH] * DEPTH + [OUT]
    return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]


def unflatten(params):
    out, k = [], 0
    for o, i in shapes():
        W = params[k:k + o * i].reshape(o, i); k += o * i
        b = params[k:k + o]; k += o
        out.append((W, b))
    assert k == len(params)
    return out


def n_params():
    return sum(o * i + o for o, i in shapes())


def forward(params, X, mu, sd, sd_out):
    """Prediction y (N, OUT) and the cache of the backward pass."""
    layers = unflatten(np.asarray(params, float))
    a = (np.asarray(X, float) - mu) / sd
    acts = [a]
    zs = []
    for li, (W, b) in enumerate(layers):
        z = a @ W.T + b
        zs.append(z)
        a = np.maximum(z, 0.0) if li < len(layers) - 1 else z
        acts.append(a)
    return a * sd_out, (acts, zs)


def loss_and_grad(params, X, T, mu, sd, sd_out):
    """Training loss (module docstring) and its gradient (flat, analytic)."""
    layers = unflatten(np.asarray(params, float))
    y, (acts, zs) = forward(params, X, mu, sd, sd_out)
    yn = acts[-1]
    tn = np.asarray(T, float) / sd_out
    N = len(X)
    diff = yn - tn
    loss = np.sum(diff ** 2) / (N * OUT)
    dz = 2.0 * diff / (N * OUT)
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        gW = dz.T @ acts[li]
        gb = dz.sum(axis=0)
        grads[li] = (gW, gb)
        if li > 0:
            da = dz @ W
            dz = da * (zs[li - 1] > 0)
    flat = np.concatenate([np.concatenate([g[0].ravel(), g[1]]) for g in grads])
    return loss, flat
