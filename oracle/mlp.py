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
Target: the body-frame correction from the block-diagonal velocity to the
solved one, R_p^T (U_p - U_pc,p) (6 values, padded to OUT = 8).

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
OUT = 8
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


def targets(theta, U, U_pc):
    """(M, OUT) body-frame corrections R_p^T (U_p - U_pc,p), zero padded."""
    R = rotation_matrix(np.asarray(theta, float))
    dU = (np.asarray(U, float) - np.asarray(U_pc, float)).reshape(-1, 6)
    T = np.zeros((len(dU), OUT))
    T[:, :3] = np.einsum("nba,nb->na", R, dU[:, :3])
    T[:, 3:6] = np.einsum("nba,nb->na", R, dU[:, 3:])
    return T


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
