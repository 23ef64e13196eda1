"""Single workloads for profilers (ncu): each case runs one small, fixed
piece of the solver's hot path a few times and exits, so that a capture of
one kernel (-k, -c) ends quickly.  Nothing here is timed.

    python -m paper_2107_10800_gb300.profile_cases product --blobs 60000 [--arith mixed|fp64|df64] [--symmetric]
    python -m paper_2107_10800_gb300.profile_cases colony --precision fp64|mixed [--steps 3] [--host-steps] [--tile 64]
    python -m paper_2107_10800_gb300.profile_cases batched [--steps 1] [--host-steps]
    python -m paper_2107_10800_gb300.profile_cases mlp [--rows 65536] [--calls 3]
    python -m paper_2107_10800_gb300.profile_cases periodic [--lattice 10 10 10] [--tol 1e-8] [--calls 3]

product: the all-pairs wall product u = M lambda on the first N blobs of the
1,000-bacteria suspension above a wall (each blob its own body, so the
product is the solver's work-queue kernel on one system), two targets per
thread and 4,096-source chunks for the mixed arithmetic, or with
--symmetric the symmetric product on tile pairs of 128; `--calls` products.
colony: Euler steps of the diatom colony (2,560 blobs, 62 sliding links,
dt = 1e-3, relative residual 1e-8); with --host-steps the Arnoldi steps are
launched from the host (per-launch timing of the product on) instead of
from the CUDA-graph loop, whose kernels profilers do not capture; --tile
fixes the symmetric product on tiles of that many blobs (the autotuner's
timings mean nothing under a profiler).
batched: steps of the 256 free-space chain suspensions in one handle
(mixed precision); --host-steps as for colony.
mlp: BF16 predictions of the learned-guess network (random weights) for
`--rows` feature rows: four tcgen05 layer launches per call.
periodic: spectral Ewald products of the bacteria in a periodic box (one
bacterium per lattice site, 360 blobs each; 10 x 10 x 10 is 360,000 blobs),
relative tolerance `--tol`, `--calls` products after the pose's pair blocks.
"""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2107_10800_gb300 import build, binding, workloads as W  # noqa: E402


def product(blobs, arith, calls, symmetric=False):
    w = W.bacteria_wall(1)
    s = binding.Solver.from_workload(w, precision="mixed")
    r = s.blobs()[:blobs]
    s.close()
    n = len(r)
    s = binding.Solver(eta=w["eta"], a=w["a"], wall=1, precision="mixed")
    s.set_bodies(r, np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)), np.arange(n + 1), np.zeros((n, 3)),
                 np.zeros((n, 6)), np.arange(n))
    if symmetric:
        s.set_mobility_layout(3, 128)
    else:
        s.set_mobility_layout(2 if arith == "mixed" else 1, 4096 if arith == "mixed" else 0)
    lam = np.random.default_rng(0).standard_normal(r.shape)
    for _ in range(calls):
        s.apply_mobility_ex(lam, arith)
    s.close()


def colony(precision, steps, host_steps=False, tile=0):
    w = W.diatom_colony(1)
    s = binding.Solver.from_workload(w, t=0.0, tol=1e-8, precision=precision)
    if tile:
        s.set_mobility_layout(3, tile)
    if host_steps:
        s.mobility_timing(True)
    for k in range(steps):
        t = k * 1e-3
        if k:
            dlp, dlq, dlpd, dlqd = w["dl"](t)
            s.set_constraints(w["body_p"], w["body_q"], dlp, dlq, dlpd, dlqd)
        s.step(t, 1e-3, dl_next=w["dl"](t + 1e-3)[:2])
    s.close()


def batched(steps, host_steps=False):
    s = binding.Solver.from_workloads(W.batched_chains(1), tol=1e-8, precision="mixed")
    if host_steps:
        s.mobility_timing(True)
    for k in range(steps):
        s.step(k * 1e-3, 1e-3)
    s.close()


def mlp(rows, calls):
    net = binding.Mlp(seed=1)
    X = np.random.default_rng(0).standard_normal((rows, binding.MLP_FEAT)).astype(np.float32)
    for _ in range(calls):
        net.predict(X, bf16=True)
    net.close()


def periodic(lattice, tol, calls):
    w = W.bacteria_periodic(5, lattice=tuple(lattice))
    s = binding.Solver.from_workload(w, ewald_tol=tol)
    lam = np.random.default_rng(6).standard_normal((s.Nb, 3))
    for _ in range(calls):
        s.apply_mobility(lam)
    s.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["product", "colony", "batched", "mlp", "periodic"])
    ap.add_argument("--lattice", type=int, nargs=3, default=[10, 10, 10])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--rows", type=int, default=65536)
    ap.add_argument("--blobs", type=int, default=60000)
    ap.add_argument("--arith", default="mixed", choices=["mixed", "fp64", "df64"])
    ap.add_argument("--calls", type=int, default=3)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--host-steps", action="store_true")
    ap.add_argument("--symmetric", action="store_true")
    ap.add_argument("--tile", type=int, default=0)
    a = ap.parse_args()
    build.build()
    if a.case == "product":
        product(a.blobs, a.arith, a.calls, a.symmetric)
    elif a.case == "colony":
        colony(a.precision, a.steps, a.host_steps, a.tile)
    elif a.case == "batched":
        batched(a.steps, a.host_steps)
    elif a.case == "periodic":
        periodic(a.lattice, a.tol, a.calls)
    else:
        mlp(a.rows, a.calls)


if __name__ == "__main__":
    main()
