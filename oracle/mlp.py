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
        R_p^T u_far(q_p)                3 values: far flow (below)
        J, row-major                    9 values: its body-frame gradient
                                        by central differences along the
                                        body axes, J_cj = (R_p^T (u_far(q_p
                                        + h R_p e_j) - u_far(q_p - h R_p
                                        e_j)))_c / 2h, h = 0.5
  and zeros up to 144; L = 4.  The far flow is the flow of point forces at
  the tracking points of the bodies of the other articulated bodies of the
  system within FAR_R of q_p: u_far(x) = sum_k M(x, q_k) f_k over bodies k
  of the same system and another articulated body with |q_k - q_p|^2 <=
  FAR_R^2, M the blob pair tensor (free or wall) with the blob radius, f_k
  the sum over k's blobs of the blob forces of the block-diagonal solution
  P~^-1 b.  (The cutoff keeps the feature's scale independent of the size
  of the suspension.)
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
from .mobility import pair_tensor

FEAT = 144
OUT = 32
NFLOW = 29
RIDGE = 1e-6
WIDTH = 256
DEPTH = 3
KNN = 16
LSCALE = 4.0
FAR_H = 0.5
FAR_R = 16.0


def far_flow(q, theta, f, system_of_body, assembly, a, eta, wall):
    """Body-frame far flow R_p^T u_far(q_p) (M, 3) and its body-frame
    central-difference gradient J (M, 3, 3), J[p, c, j] = d u_c / d x_j
    along body axis j (module docstring)."""
    q = np.asarray(q, float)
    R = rotation_matrix(np.asarray(theta, float))
    f = np.asarray(f, float).reshape(-1, 3)
    sysb = np.asarray(system_of_body)
    asm = np.asarray(assembly)
    M = len(q)
    u = np.zeros((M, 7, 3))
    for p in range(M):
        d2 = np.sum((q - q[p]) ** 2, axis=1)
        src = np.nonzero((sysb == sysb[p]) & (asm != asm[p]) & (d2 <= FAR_R ** 2))[0]
        if len(src) == 0:
            continue
        steps = np.zeros((7, 3))
        for j in range(3):
            steps[1 + 2 * j] = FAR_H * R[p][:, j]
            steps[2 + 2 * j] = -FAR_H * R[p][:, j]
        x = q[p] + steps  # (7, 3) evaluation points
        T = pair_tensor(x[:, None, :], q[src][None, :, :], a, eta, wall)  # (7, S, 3, 3)
        u[p] = np.einsum("esab,sb->ea", T, f[src]) @ R[p]  # rows R_p^T u
    J = np.stack([(u[:, 1 + 2 * j] - u[:, 2 + 2 * j]) / (2 * FAR_H) for j in range(3)], axis=2)
    return u[:, 0], J


def features(q, theta, F, blob_offset, U_pc, system_of_body, wall, lam_pc, assembly, a, eta):
    """(M, FEAT) features of every body (see module docstring); lam_pc
    (3Nb) are the blob forces of the block-diagonal solution."""
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
    off = np.asarray(blob_offset)
    lam = np.asarray(lam_pc, float).reshape(-1, 3)
    f = np.stack([lam[off[k]:off[k + 1]].sum(axis=0) for k in range(M)]) if M else np.zeros((0, 3))
    u, J = far_flow(q, theta, f, system_of_body, assembly, a, eta, wall)
    fb = 7 * KNN + 14
    X[:, fb:fb + 3] = u
    X[:, fb + 3:fb + 12] = J.reshape(M, 9)
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
