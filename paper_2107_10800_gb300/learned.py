"""Training pipeline of the learned initial guess (the paper has no learned
component).  Every step runs in the library: the solves that make the
training targets, the feature kernel, FP32 training and the BF16 inference
the solver uses; this module only chooses workloads and seeds and moves
arrays.

Data: bacteria above a wall (the head-flagellum model of Sec. 4.3 and 5.2)
in small suspensions at the lateral density of the large one, several poses
per suspension (time steps of Sec. 4.3), solved to a tight tolerance; each
body gives one sample (features, body-frame fit of the background flow that
the other bodies induce at its blobs).
"""
import math

import numpy as np

from . import binding, workloads

# Lateral density of the 1,000-bacteria suspension: 1000 / 250^2.
DENSITY = 1000.0 / 250.0 ** 2


def bacteria_at_density(seed, n_bact):
    """Bacteria above a wall in a square holding them at DENSITY."""
    box = math.sqrt(n_bact / DENSITY)
    return workloads.bacteria_wall(seed, n_bact=n_bact, box=box)


def collect(seeds, n_bact=24, poses=2, dt=0.05, systems_per_handle=32, tol=1e-9,
            precision="mixed"):
    """Features and targets of every body of the suspensions `seeds`, at
    `poses` poses each (the initial one and poses-1 Euler steps of dt).
    Returns X (N x 144), T (N x 32) as float32."""
    Xs, Ts = [], []
    for k0 in range(0, len(seeds), systems_per_handle):
        ws = [bacteria_at_density(s, n_bact) for s in seeds[k0:k0 + systems_per_handle]]
        solver = binding.Solver.from_workloads(ws, precision=precision, tol=tol, max_iter=2000)
        try:
            for p in range(poses):
                solver.solve()
                X, T = solver.learned_features(targets=True)
                Xs.append(X)
                Ts.append(T)
                if p + 1 < poses:
                    solver.step(p * dt, dt)
        finally:
            solver.close()
    return np.concatenate(Xs), np.concatenate(Ts)


def normalisation(X, T):
    """Per-feature mean and spread (spread 1 for constant columns) and the
    per-output spread (1 for the padded outputs)."""
    mu = X.mean(axis=0)
    sd = X.std(axis=0)
    sd = np.where(sd > 1e-6, sd, 1.0)
    sdo = np.sqrt((T ** 2).mean(axis=0))
    sdo = np.where(sdo > 1e-12, sdo, 1.0)
    return mu.astype(np.float32), sd.astype(np.float32), sdo.astype(np.float32)


def train(X, T, epochs=40, batch=256, lr=1e-3, seed=0, stream=None):
    """A trained binding.Mlp and its final training loss."""
    mlp = binding.Mlp(seed=seed, stream=stream)
    mu, sd, sdo = normalisation(X, T)
    mlp.set_norm(mu, sd, sdo)
    loss = mlp.train(X, T, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return mlp, loss


def cold_start_iterations(ws, mlp, precision="fp64", tol=1e-8, check=True):
    """GMRES iterations and relative residuals of the cold-start solve of the
    workloads ws (one handle, one system each) from P~^-1 b and from the
    learned guess."""
    out = {}
    for name, model in (("block_diagonal", None), ("learned", mlp)):
        solver = binding.Solver.from_workloads(ws, precision=precision, tol=tol, max_iter=2000)
        try:
            if model is not None:
                solver.set_learned(model, check=check)
            _, _, _, st = solver.solve()
            out[name] = {k: st[k] for k in ("iterations", "rel_residual", "rel_residual0",
                                            "ms_gmres", "learned_systems")}
        finally:
            solver.close()
    return out
