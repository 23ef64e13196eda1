"""Benchmark of the constrained mobility solve: one time step of the diatom
colony above a no-slip wall (32 rods x 80 blobs = 2,560 blobs, 62 sliding
links, dt = 1e-3, plain FP64, GMRES to relative residual 1e-8).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one am_solve_step: pose, preconditioner build, warm-started GMRES
solve, Euler update, reconstruction and correction.  The headline metric is
blob-pair interactions of the mobility products per second over the whole
step (pairs evaluated / step time).  Prints one JSON line (rank 0).

With N > 1 (torchrun) every rank runs its own colony (seed 1 + rank): the
suspensions are independent, so there is no exchange and scaling is weak.
--impl reference times the FP64 CPU oracle on the same workload (a bounded
sample of mobility rows per step), rank 0 only.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RPY pair-interactions/s"
UNIT = "pairs/s"
DT = 1e-3
TOL = 1e-8
WORKLOAD = ("diatom colony above a no-slip wall: 32 rods of 2x40 blobs (2,560 blobs, a=0.1), "
            "62 sliding links, dt=1e-3, FP64, GMRES relative residual 1e-8")
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2
# DRAM bytes (read + write) of one launch of the wall product on this colony
# per (precision, symmetric tile), from ncu captures of the colony's steps
# with the tile fixed (profile_cases colony --host-steps --tile T;
# dram__bytes_read.sum + dram__bytes_write.sum); absent where no capture of
# the kernel as it now stands exists
TRAFFIC_BYTES = {("fp64", 32): 337152, ("fp64", 64): 219648}
# flop per unordered pair of the symmetric FP64 wall product (see run_ours)
SYM_WALL_FLOP_PER_UNORDERED_PAIR = 126


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running,
    written to $AM_CLOCK_DIR/clocks_rank<gpu>.csv (default: the temporary
    directory)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            d = os.environ.get("AM_CLOCK_DIR") or tempfile.gettempdir()
            os.makedirs(d, exist_ok=True)
            self.path = os.path.join(d, "clocks_rank%d.csv" % self.gpu)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except Exception:
            return None
    return None


def _oracle_rows_job(args):
    """One worker's share of the oracle's mobility rows (spawned process)."""
    r, lam, rows, a, eta, wall = args
    from oracle import mobility as om
    om.mobility_rows(r, lam, rows, a, eta, wall)
    return len(rows)


class OraclePool:
    """The host cores for the oracle: one single-threaded worker process per
    core (spawned, so none inherits a CUDA context), each computing the
    oracle's mobility rows for its share of the sampled targets.  The oracle
    itself is unchanged; this only runs it on every core."""

    def __init__(self, procs=None):
        import multiprocessing as mp
        self.procs = procs or os.cpu_count() or 1
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(v, "1")
        self.pool = mp.get_context("spawn").Pool(self.procs)
        # workers import the oracle on their first job
        r = np.zeros((4, 3)); r[:, 0] = np.arange(4); r[:, 2] = 1.0
        self.pool.map_async(_oracle_rows_job, [(r, r, np.arange(1), 0.1, 1.0, 0)] * self.procs).get(300)

    def rows(self, r, lam, rows, a, eta, wall):
        """Wall time of the oracle's rows `rows`, split over the workers."""
        parts = [p for p in np.array_split(np.asarray(rows), self.procs) if len(p)]
        t0 = time.perf_counter()
        self.pool.map_async(_oracle_rows_job, [(r, lam, p, a, eta, wall) for p in parts]).get(600)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_sample(w, t, pool, seconds=10.0):
    """The oracle's mobility rows on a bounded sample of target blobs of the
    workload, on all workers of `pool`: returns (pairs/s, pairs, rows,
    elapsed)."""
    from oracle.system import System
    S = System(w, t=t)
    lam = np.random.default_rng(0).standard_normal((S.Nb, 3))
    rng = np.random.default_rng(1)
    probe = rng.choice(S.Nb, min(S.Nb, 4 * pool.procs), replace=False)
    per_row = pool.rows(S.r, lam, probe, S.a, S.eta, S.wall) / len(probe)
    nrows = int(min(S.Nb, max(len(probe), seconds / max(per_row, 1e-7))))
    rows = rng.choice(S.Nb, nrows, replace=False)
    el = pool.rows(S.r, lam, rows, S.a, S.eta, S.wall)
    pairs = nrows * S.Nb
    return pairs / el, pairs, nrows, el


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from paper_2107_10800_gb300 import workloads as W
    w = W.diatom_colony(1)
    nb = W.counts(w)[0]
    pool = OraclePool()
    for _ in range(args.warmup):
        oracle_sample(w, 0.0, pool, seconds=0.5)
    times, pairs_tot = [], 0
    per_step = max(1.0, min(10.0, 120.0 / max(args.steps, 1)))
    for k in range(args.steps):
        rate, pairs, nrows, el = oracle_sample(w, k * DT, pool, seconds=per_step)
        times.append(el)
        pairs_tot += pairs
    pool.close()
    value = pairs_tot / sum(times)
    sample = ("oracle mobility rows of the colony (all %d target blobs x %d sources is one product), "
              "a sample of target rows per step split over %d worker processes" % (nb, nb, pool.procs))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "blobs": nb},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def matvec_at_scale(torch, binding, W, stream, fp32_peak, fp64_peak):
    """The solver's all-pairs wall product at the bacteria-suspension scale
    (1,000 bacteria, 360,000 blobs, a = 0.05): the mixed work-queue kernel
    with two targets per thread in paired FP32 lanes and 4,096-source chunks
    on all blobs, and the symmetric mixed product (tile pairs of 128), the FP64 kernels (one-direction and symmetric, tiles of
    128) on the first 40,000 (an FP64 product on all blobs takes about 20 s).  The blobs are single-blob bodies of one
    handle; kernel time from CUDA events around each launch
    (am_mobility_timing), after a warm-up product."""
    w = W.bacteria_wall(1)
    s = binding.Solver.from_workload(w, precision="mixed")
    R = s.blobs()
    s.close()
    out = {"workload": "bacteria above a wall: 1,000 x (200-blob head + 16 x 10-blob flagellum), "
                       "360,000 blobs, a=0.05"}
    fpp = binding.flops_per_pair(1)
    for key, prec, n, layout, peak in (("mixed", "mixed", len(R), (2, 4096), fp32_peak),
                                       ("mixed_symmetric", "mixed", len(R), (3, 128), fp32_peak),
                                       ("fp64", "fp64", 40_000, (1, 0), fp64_peak),
                                       ("fp64_symmetric", "fp64", 40_000, (3, 128), fp64_peak)):
        r = R[:n]
        s = binding.Solver(eta=w["eta"], a=w["a"], wall=1, precision=prec)
        s.set_bodies(r, np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)), np.arange(n + 1), np.zeros((n, 3)),
                     np.zeros((n, 6)), np.arange(n))
        s.set_mobility_layout(*layout)
        lam = np.random.default_rng(0).standard_normal(r.shape)
        s.apply_mobility_ex(lam, prec)  # warm-up
        s.mobility_timing(True)
        for _ in range(2 if key == "mixed" else 1):
            s.apply_mobility_ex(lam, prec)
        ms, launches = s.mobility_timing(False)
        s.close()
        t = ms * 1e-3 / max(launches, 1)
        pairs = float(n) * n
        out[key] = {"blobs": n, "ms": t * 1e3, "pairs_per_s": pairs / t,
                    "tflops": pairs * fpp / t / 1e12, "frac_of_fma_peak": pairs * fpp / t / peak,
                    "kernel": {"mixed": "rpy_items_mixed_x2<wall>", "mixed_symmetric": "rpy_sym_mixed_x2<wall>",
                               "fp64": "rpy_items_f64<wall>", "fp64_symmetric": "rpy_sym_f64<wall, tile 128>"}[key]}
    return out


def steric_at_scale(binding, W, reps=3):
    """The steric repulsion (soft potential between bacteria, cutoff 2a +
    8 b with b = a, and the wall term) on the 1,000-bacteria suspension:
    host time of am_steric_forces (pose, pair search, body sums, 8.6 MB of
    forces back to the host), median of `reps` calls after a warm-up."""
    w = W.bacteria_wall(1)
    s = binding.Solver.from_workload(w, precision="mixed")
    a = w["a"]
    s.set_repulsion(0.1, a, 2 * a + 8 * a, 0.1, a)
    s.steric_forces()
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        f = s.steric_forces()
        ts.append(time.perf_counter() - t0)
    s.close()
    return {"workload": "1,000 bacteria, 360,000 blobs above a wall; cutoff 10a",
            "ms": 1e3 * statistics.median(ts), "blobs_with_force": int(np.count_nonzero(np.abs(f).sum(axis=1)))}


def products_compared(binding, W, fp32_peak, fp64_peak, n=60_000):
    """The three pair arithmetics of the solver on the same blobs (the first
    n blobs of the bacteria suspension, as single-blob bodies of one
    handle): FP64, double-float (the mixed solver's outer residual) and
    mixed FP32.  Kernel time from CUDA events around each launch of the
    all-pairs kernel (am_mobility_timing), second call of each."""
    w = W.bacteria_wall(1)
    s = binding.Solver.from_workload(w, precision="mixed")
    r = s.blobs()[:n]
    s.close()
    s = binding.Solver(eta=w["eta"], a=w["a"], wall=1, precision="mixed")
    th = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    s.set_bodies(r, th, np.arange(n + 1), np.zeros((n, 3)), np.zeros((n, 6)), np.arange(n))
    lam = np.random.default_rng(0).standard_normal(r.shape)
    fpp = binding.flops_per_pair(1)
    out = {"workload": "first %d blobs of the 1,000-bacteria suspension above a wall" % n}
    ref = None
    for arith in ("fp64", "df64", "mixed"):
        s.apply_mobility_ex(lam, arith)  # warm-up (and autotuning on the first call)
        s.mobility_timing(True)
        u = s.apply_mobility_ex(lam, arith)
        ms, launches = s.mobility_timing(False)
        if ref is None:
            ref = u
        err = float(np.abs(u - ref).max() / np.abs(ref).max())
        t = ms * 1e-3 / max(launches, 1)
        pairs = float(n) * n
        peak = fp64_peak if arith == "fp64" else fp32_peak
        out[arith] = {"ms": ms / max(launches, 1), "pairs_per_s": pairs / t,
                      "tflops_algorithmic": pairs * fpp / t / 1e12,
                      "frac_of_fma_peak": pairs * fpp / t / peak,
                      "max_rel_diff_vs_fp64": err}
    s.close()
    return out


def learned_form(binding, W):
    """The learned initial guess: a network trained on the GPU (suspensions
    of 32 bacteria, seeds 1000-1047, two poses each: 52,224 samples, 20
    epochs), then cold-start solves at relative residual 1e-8 on held-out
    suspensions: 556 bacteria (200,160 blobs; mixed precision) from P~^-1 b
    and from the learned guess, and 100 bacteria (36,000 blobs) in plain FP64,
    mixed, and mixed with the learned guess.  Host wall time of the second
    am_solve of each handle (every am_solve starts cold; the first one also
    tunes the product layout)."""
    from paper_2107_10800_gb300 import learned
    t0 = time.perf_counter()
    X, T = learned.collect(list(range(1000, 1048)), n_bact=32, poses=2, systems_per_handle=16)
    t1 = time.perf_counter()
    net, loss = learned.train(X, T, epochs=20, batch=256, lr=1e-3, seed=0)
    t2 = time.perf_counter()
    out = {"training": {"samples": int(len(X)), "final_loss": loss, "collect_s": t1 - t0,
                        "train_s": t2 - t1}}

    def run(w, precision, model):
        s = binding.Solver.from_workload(w, precision=precision, tol=1e-8, max_iter=2000)
        if model is not None:
            s.set_learned(model, check=True)
        s.solve()  # warm-up: autotuning of the product layout (every am_solve starts cold)
        tt = time.perf_counter()
        _, _, _, st = s.solve()
        wall = time.perf_counter() - tt
        s.close()
        return {"solve_ms": 1e3 * wall, "iterations": st["iterations"],
                "rel_residual0": st["rel_residual0"], "rel_residual": st["rel_residual"],
                "learned_systems": st["learned_systems"]}

    out["held_out_100"] = learned_held_out(binding, learned, net)
    big = learned.bacteria_at_density(20100, 556)
    out["bacteria_556"] = {"blobs": int(big["blob_offset"][-1]),
                           "mixed_block_diagonal_start": run(big, "mixed", None),
                           "mixed_learned_start": run(big, "mixed", net)}
    small = learned.bacteria_at_density(20200, 100)
    out["bacteria_100"] = {"blobs": int(small["blob_offset"][-1]),
                           "fp64": run(small, "fp64", None),
                           "mixed": run(small, "mixed", None),
                           "mixed_learned_start": run(small, "mixed", net)}
    net.close()
    return out


def learned_held_out(binding, learned, net, seeds=range(20300, 20320), n_bact=100):
    """Cold-start solves of held-out suspensions of 100 bacteria (36,000
    blobs, mixed precision, relative residual 1e-8), one handle per seed and
    start, with the product layout fixed (one target per thread, source
    chunks chosen for the size) so both starts run the same kernels: GMRES
    iterations, initial relative residual and host wall time of the solve,
    per seed and as mean and standard deviation."""
    res = {"plain": [], "learned": []}
    for seed in seeds:
        w = learned.bacteria_at_density(seed, n_bact)
        for name, model in (("plain", None), ("learned", net)):
            s = binding.Solver.from_workload(w, precision="mixed", tol=1e-8, max_iter=2000)
            s.set_mobility_layout(1, 0)
            if model is not None:
                s.set_learned(model, check=True)
            t0 = time.perf_counter()
            _, _, _, st = s.solve()
            ms = 1e3 * (time.perf_counter() - t0)
            s.close()
            res[name].append((st["iterations"], st["rel_residual0"], ms, st["rel_residual"]))

    def stats(v):
        a = np.array(v, dtype=float)
        return {"mean": float(a.mean()), "std": float(a.std())}

    out = {"workload": "%d held-out suspensions of %d bacteria above a wall (seeds %d-%d), mixed, "
                       "cold start, relative residual 1e-8" % (len(seeds), n_bact, seeds[0], seeds[-1])}
    for name in ("plain", "learned"):
        r = res[name]
        out[name] = {"iterations": stats([x[0] for x in r]), "rel_residual0": stats([x[1] for x in r]),
                     "solve_ms": stats([x[2] for x in r]), "max_rel_residual": max(x[3] for x in r)}
    d = [l[0] - p[0] for p, l in zip(res["plain"], res["learned"])]
    out["iteration_change_per_seed"] = d
    out["iteration_change"] = stats(d)
    return out


def rk2_form(binding, W, steps=5, warmup=2):
    """The explicit midpoint (RK2) step on the bench colony: two solves, two
    reconstructions and corrections per step, FP64 and mixed, relative
    residual 1e-8.  Host wall time per step (each call ends with the outputs
    on the host), after warm-up steps."""
    out = {"workload": WORKLOAD.replace("FP64, ", "") + ", explicit midpoint step"}
    for prec in ("fp64", "mixed"):
        w = W.diatom_colony(1)
        s = binding.Solver.from_workload(w, t=0.0, tol=TOL, precision=prec)
        times, iters, resid = [], [], []
        for k in range(warmup + steps):
            t = k * DT
            if k:
                dlp, dlq, dlpd, dlqd = w["dl"](t)
                s.set_constraints(w["body_p"], w["body_q"], dlp, dlq, dlpd, dlqd)
            t0 = time.perf_counter()
            _, _, _, st = s.step_rk2(t, DT, dl_half=w["dl"](t + 0.5 * DT), dl_next=w["dl"](t + DT)[:2])
            if k >= warmup:
                times.append(time.perf_counter() - t0)
                iters.append(st["iterations"])
                resid.append(st["rel_residual"])
        s.close()
        out[prec] = {"ms_per_step": 1e3 * statistics.mean(times), "gmres_iterations_per_step": statistics.mean(iters),
                     "max_rel_residual": max(resid)}
    return out


def guess_form(binding, W, steps=8, warmup=3):
    """The bench colony's Euler step with the initial guess of each solve
    taken from the solution history (am_set_initial_guess): order 1 = the
    previous solution (the headline's), 2 and 3 = the extrapolation in time
    through the last 2 or 3 solutions; FP64 and mixed, relative residual
    1e-8.  Host wall time per step after warm-up steps."""
    out = {"workload": WORKLOAD.replace("FP64, ", "") + ", Euler step, initial guess from the history"}
    for prec in ("fp64", "mixed"):
        res = {}
        for order in (1, 2, 3):
            w = W.diatom_colony(1)
            s = binding.Solver.from_workload(w, t=0.0, tol=TOL, precision=prec)
            s.set_initial_guess(order)
            times, iters, resid, r0 = [], [], [], []
            for k in range(warmup + steps):
                t = k * DT
                if k:
                    dlp, dlq, dlpd, dlqd = w["dl"](t)
                    s.set_constraints(w["body_p"], w["body_q"], dlp, dlq, dlpd, dlqd)
                t0 = time.perf_counter()
                _, _, _, st = s.step(t, DT, dl_next=w["dl"](t + DT)[:2])
                if k >= warmup:
                    times.append(time.perf_counter() - t0)
                    iters.append(st["iterations"])
                    resid.append(st["rel_residual"])
                    r0.append(st["rel_residual0"])
            s.close()
            res["order_%d" % order] = {"ms_per_step": 1e3 * statistics.mean(times),
                                       "gmres_iterations_per_step": statistics.mean(iters),
                                       "initial_rel_residual": statistics.mean(r0),
                                       "max_rel_residual": max(resid)}
        out[prec] = res
    return out


def single_blob_form(binding, W, steps=3, warmup=2):
    """Single-blob bodies with rotational coupling (free space): 400
    filaments of 15 spheres (a = 0.5, neighbours 1.05 apart, ball joints),
    6,000 bodies, 52,800 unknowns, FP64, relative residual 1e-8; host time
    per Euler step after warm-up steps."""
    w = W.chains_free_space(1, n_chains=400, bodies_per_chain=15, box=10.0 * 100 ** (1.0 / 3.0))
    w = dict(w, a=0.5)
    s = binding.Solver.from_workload(w, tol=TOL, single_blob=True)
    times, iters = [], []
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        _, _, _, st = s.step(k * DT, DT)
        if k >= warmup:
            times.append(time.perf_counter() - t0)
            iters.append(st["iterations"])
    s.close()
    M = len(w["q"])
    return {"workload": "400 free-space filaments of 15 single-blob spheres (a=0.5), ball joints",
            "bodies": M, "unknowns": 6 * M + 3 * len(w["body_p"]), "ms_per_step": 1e3 * statistics.mean(times),
            "gmres_iterations_per_step": statistics.mean(iters), "max_rel_residual": st["rel_residual"]}


def batched_form(torch, binding, W, stream, steps=2):
    """One handle holding the 256 free-space chain suspensions (blob counts
    log-uniform in [500, 20,000], 1.41 M blobs), mixed precision, solved
    together: time per step of the whole batch (after one warm-up step)."""
    ws = W.batched_chains(1)
    t0 = time.perf_counter()
    s = binding.Solver.from_workloads(ws, tol=1e-8, precision="mixed", stream=stream.cuda_stream)
    q, th = s.bodies(0)  # builds the device layout of all systems
    setup_s = time.perf_counter() - t0
    s.step(0.0, 1e-3)
    out = []
    for k in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        U, phi, lam, st = s.step((k + 1) * 1e-3, 1e-3)
        e1.record(stream)
        torch.cuda.synchronize()
        out.append((e0.elapsed_time(e1), st))
    ms = statistics.mean(o[0] for o in out)
    st = out[-1][1]
    s.close()
    return {"workload": "256 free-space chain suspensions, blob counts log-uniform in [500, 20,000] "
                        "(1,410,840 blobs, 117,570 bodies), mixed precision, one handle",
            "ms_per_step": ms, "pairs_per_s": st["pairs"] / (ms * 1e-3),
            "gmres_iterations": st["iterations"], "max_rel_residual": st["rel_residual"],
            "ms_precond": st["ms_precond"], "ms_gmres": st["ms_gmres"], "setup_s": setup_s}


def chains_solve(torch, binding, W, stream, reps=20, warmup=3):
    """The small latency-bound case: 4 free-space chains of 8 icosahedral
    shells (384 blobs, 28 ball joints, 1,428 unknowns), plain FP64, one
    GMRES solve at relative residual 1e-10 per call (am_solve: pose,
    preconditioner build, solve, outputs to the host).  Device time (CUDA
    events on the solver's stream) and host wall time per solve, after
    warm-up solves; every am_solve starts cold (no history)."""
    w = W.chains_free_space(1)
    s = binding.Solver.from_workload(w, tol=1e-10, precision="fp64", stream=stream.cuda_stream)
    for _ in range(warmup):
        s.solve()
    dev, host, its = [], [], []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0.record(stream)
        _, _, _, st = s.solve()
        e1.record(stream)
        torch.cuda.synchronize()
        host.append(time.perf_counter() - t0)
        dev.append(e0.elapsed_time(e1))
        its.append(st["iterations"])
    s.close()
    nb, M, P, n = W.counts(w)
    return {"workload": "4 free-space chains of 8 icosahedral 12-blob shells (a=0.1), ball joints; "
                        "FP64, one solve at relative residual 1e-10",
            "blobs": nb, "unknowns": n, "us_per_solve": 1e3 * statistics.median(dev),
            "us_per_solve_host": 1e6 * statistics.median(host), "gmres_iterations": statistics.median(its),
            "max_rel_residual": st["rel_residual"]}


def bacteria_step(torch, binding, W, stream, dt=1e-3, rows=4096):
    """The 1,000-bacteria suspension above a wall (360,000 blobs, 17,000
    bodies, 17,000 links), mixed form: a first Euler step from the
    block-diagonal guess (it also tunes the product layout), then one timed
    Euler step warm-started from the first step's solution (CUDA events on
    the solver's stream; the step includes pose, preconditioner build,
    solve to relative residual 1e-8 judged on the double-float residual,
    update, reconstruction and correction; the reported relative residual is
    the double-float one or, when the last correction was computed from a
    double-float residual, the inner solve's mixed residual plus a bound on
    the mixed product's error: an upper bound either way).  Then the mixed
    product against
    the FP64 product on `rows` sampled target rows (four blocks of
    contiguous blobs against all 360,000 sources) at the stepped pose."""
    w = W.bacteria_wall(1)
    s = binding.Solver.from_workload(w, tol=1e-8, precision="mixed", max_iter=1000, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, _, st0 = s.step(0.0, dt)
    first_s = time.perf_counter() - t0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    _, _, _, st = s.step(dt, dt)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    r = s.blobs()
    n = len(r)
    lam = np.random.default_rng(5).standard_normal(r.shape)
    u_mixed = s.apply_mobility(lam)
    s.close()
    dev = torch.device("cuda")
    dr = torch.tensor(r, device=dev)
    dl = torch.tensor(lam, device=dev)
    starts = np.random.default_rng(6).choice(n - rows // 4, 4, replace=False)
    err = 0.0
    with torch.cuda.stream(stream):
        for r0 in starts:
            nr = rows // 4
            du = torch.empty((nr, 3), dtype=torch.float64, device=dev)
            nbytes = binding.rpy_matvec_rows_workspace(n, nr, "fp64")
            work = torch.empty(nbytes // 8 + 64, dtype=torch.float64, device=dev)
            aligned = (work.data_ptr() + 255) // 256 * 256
            binding.rpy_matvec_rows_ptr(dr.data_ptr(), dl.data_ptr(), du.data_ptr(), n, int(r0), nr, w["eta"],
                                        w["a"], 1, "fp64", aligned, nbytes, stream.cuda_stream)
            stream.synchronize()
            ref = du.cpu().numpy()
            err = max(err, float(np.abs(u_mixed[r0:r0 + nr] - ref).max() / np.abs(ref).max()))
    return {"workload": "1,000 bacteria above a wall: 200-blob head + 16 x 10-blob flagellum each, 360,000 "
                        "blobs, 17,000 bodies, 17,000 links, a=0.05; mixed precision, dt=%g" % dt,
            "ms_per_step": ms, "gmres_iterations": st["iterations"], "rel_residual": st["rel_residual"],
            "constraint_residual": st["constraint_residual"], "ms_precond": st["ms_precond"],
            "ms_gmres": st["ms_gmres"], "pairs_per_s": st["pairs"] / (ms * 1e-3),
            "first_step": {"s_host": first_s, "gmres_iterations": st0["iterations"],
                           "rel_residual": st0["rel_residual"]},
            "mixed_vs_fp64_product_rows": {"rows": rows, "max_rel_diff": err}}


def periodic_form(torch, binding, W, stream, products=5):
    """Fast summation: the 1,000 bacteria in a triply periodic 150 x 30 x 30
    box (360,000 blobs, aligned on a jittered lattice), FP64 spectral Ewald
    product (csrc/periodic.cu).  Per tolerance 1e-8 and 1e-10: the product's
    device time (CUDA events around each product launch, am_mobility_timing,
    after the pose's pair blocks) and its parameters; then one solve at
    relative residual 1e-8 with the 1e-10 product (pose, pair blocks,
    preconditioner build, GMRES) and one Euler step after it, CUDA events on
    the solver's stream; then the mixed form (FP32 products inside, FP64
    outer residuals): its FP32 product and one solve at 1e-8."""
    w = W.bacteria_periodic(5)
    lam = np.random.default_rng(6).standard_normal((int(w["blob_offset"][-1]), 3))
    out = {"workload": "1,000 bacteria (360 blobs each, a=0.05) on a jittered 10 x 10 x 10 lattice in a "
                       "triply periodic 150 x 30 x 30 box, 360,000 blobs; FP64 spectral Ewald product"}
    for tol in (1e-8, 1e-10):
        s = binding.Solver.from_workload(w, ewald_tol=tol, stream=stream.cuda_stream)
        s.apply_mobility(lam)  # pair blocks of the pose
        s.mobility_timing(True)
        for _ in range(products):
            s.apply_mobility(lam)
        ms, k = s.mobility_timing(False)
        info = s.periodic_info()
        s.close()
        out["product_tol_%g" % tol] = {"ms": ms / max(k, 1), "grid": list(info["grid"]),
                                       "window_points": info["support"], "xi": info["xi"], "r_c": info["r_c"],
                                       "real_space_pairs": info["real_pairs"]}
    s = binding.Solver.from_workload(w, tol=1e-8, ewald_tol=1e-10, stream=stream.cuda_stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    _, _, _, st = s.solve()
    e1.record(stream)
    torch.cuda.synchronize()
    solve_ms = e0.elapsed_time(e1)
    e0.record(stream)
    _, _, _, st2 = s.step(0.0, 1e-3)
    e1.record(stream)
    torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1)
    s.close()
    out.update({"solve_ms": solve_ms, "gmres_iterations": st["iterations"], "rel_residual": st["rel_residual"],
                "ms_precond": st["ms_precond"], "ms_gmres": st["ms_gmres"], "step_ms": step_ms,
                "step_gmres_iterations": st2["iterations"], "step_rel_residual": st2["rel_residual"]})
    # mixed: FP32 wave part and blocks inside, FP64 product for the outer residuals
    s = binding.Solver.from_workload(w, tol=1e-8, ewald_tol=1e-10, precision="mixed", stream=stream.cuda_stream)
    s.apply_mobility(lam)
    s.mobility_timing(True)
    for _ in range(products):
        s.apply_mobility_ex(lam, "mixed")
    ms32, k32 = s.mobility_timing(False)
    torch.cuda.synchronize()
    e0.record(stream)
    _, _, _, st3 = s.solve()
    e1.record(stream)
    torch.cuda.synchronize()
    s.close()
    out["mixed"] = {"product_ms": ms32 / max(k32, 1), "solve_ms": e0.elapsed_time(e1),
                    "gmres_iterations": st3["iterations"], "rel_residual": st3["rel_residual"],
                    "ms_precond": st3["ms_precond"], "ms_gmres": st3["ms_gmres"]}
    return out


def combine_ranks(torch, total_s, pairs, e2e_ms_mean, steps, device):
    """Whole-job figures over the ranks of the process group: the timed
    region is the slowest rank's, the pairs are all ranks' (independent
    suspensions, weak scaling).  Returns (seconds, pairs, end-to-end pairs/s
    per step at the slowest rank's end-to-end step time)."""
    tt = torch.tensor([total_s, float(pairs), e2e_ms_mean], dtype=torch.float64, device=device)
    tmax = tt.clone()
    torch.distributed.all_reduce(tmax, op=torch.distributed.ReduceOp.MAX)
    tsum = tt.clone()
    torch.distributed.all_reduce(tsum, op=torch.distributed.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[1]), float(tsum[1]) / steps / (float(tmax[2]) * 1e-3)


def rank_workload(W, rank):
    """The colony of one rank: seed 1 + rank (independent suspensions)."""
    return W.diatom_colony(1 + rank)


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2107_10800_gb300 import build as _b
    from paper_2107_10800_gb300 import binding, workloads as W
    if rank == 0 or world == 1:
        _b.build()
    if world > 1:
        torch.distributed.barrier()
    _b.build()
    L = binding.lib()
    w = rank_workload(W, rank)
    nb, M, P, n = W.counts(w)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    solver = binding.Solver.from_workload(w, t=0.0, tol=TOL, precision=args.precision,
                                          stream=stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def do_step(k, outputs):
        t = k * DT
        dlp, dlq, dlpd, dlqd = w["dl"](t)
        solver.set_constraints(w["body_p"], w["body_q"], dlp, dlq, dlpd, dlqd)
        nxt = w["dl"](t + DT)[:2]
        if outputs:
            return solver.step(t, DT, dl_next=nxt)
        st = binding.StepStats()
        import ctypes
        a1 = np.ascontiguousarray(nxt[0]).ravel()
        a2 = np.ascontiguousarray(nxt[1]).ravel()
        rc = L.am_solve_step(solver.h, t, DT, a1.ctypes.data_as(binding._dp),
                             a2.ctypes.data_as(binding._dp), ctypes.byref(st), None, None, None)
        if rc not in (0, binding.AM_ERR_NOT_CONVERGED):
            raise binding.AmError(rc, L.am_last_error(solver.h).decode())
        return None, None, None, st.as_dict()

    k = 0
    for _ in range(args.warmup):
        do_step(k, False)
        k += 1
    # peaks for the roofline of the all-pairs kernel (ALU bound)
    fp64_peak = binding.alu_peak(True)
    fp32_peak = binding.alu_peak(False)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms, pairs, iters, resid, precond_ms = [], 0, [], [], []
    launches0 = binding.kernel_launches()
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(float(k))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            _, _, _, st = do_step(k, False)
            e1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            pairs += st["pairs"]
            precond_ms.append(st["ms_precond"])
            iters.append(st["iterations"])
            resid.append(st["rel_residual"])
            k += 1
        t_wall = time.perf_counter() - t_wall0
    launches = binding.kernel_launches() - launches0
    # second pass: the same steps with CUDA events around every launch of the
    # all-pairs kernel (the Arnoldi steps are then host-launched instead of
    # running in the graph loop); gives the kernel's average launch time
    solver.mobility_timing(True)
    for _ in range(min(args.steps, 5)):
        do_step(k, False)
        k += 1
    mob_ms, mob_launches = solver.mobility_timing(False)
    total_s = sum(step_ms) * 1e-3
    local_rate = pairs / total_s
    # end to end: host link schedule in, solution out, every step
    e2e_ms = []
    for _ in range(max(3, args.steps // 2)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        flush.fill_(float(k))
        torch.cuda.synchronize()
        e0.record(stream)
        U, phi, lam, st = do_step(k, True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
        k += 1
    e2e_rate = st["pairs"] / (statistics.mean(e2e_ms) * 1e-3)

    if world > 1:
        total_s_all, pairs_all, e2e_rate = combine_ranks(torch, total_s, pairs, statistics.mean(e2e_ms),
                                                         args.steps, "cuda")
    else:
        total_s_all = total_s
        pairs_all = float(pairs)
    value = pairs_all / total_s_all
    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
        return

    at_scale = matvec_at_scale(torch, binding, W, stream, fp32_peak, fp64_peak)
    compared = products_compared(binding, W, fp32_peak, fp64_peak) if world == 1 else None
    steric = steric_at_scale(binding, W) if world == 1 else None
    batched = batched_form(torch, binding, W, stream) if world == 1 else None
    learned_res = learned_form(binding, W) if world == 1 else None
    rk2_res = rk2_form(binding, W) if world == 1 else None
    guess_res = guess_form(binding, W) if world == 1 else None
    sb_res = single_blob_form(binding, W) if world == 1 else None
    chains_res = chains_solve(torch, binding, W, stream) if world == 1 else None
    periodic_res = periodic_form(torch, binding, W, stream) if world == 1 else None
    bact_res = bacteria_step(torch, binding, W, stream) if world == 1 else None
    fpp = binding.flops_per_pair(1)
    avg_launch_s = (mob_ms * 1e-3) / max(mob_launches, 1)
    achieved = nb * nb * fpp / avg_launch_s
    layout = solver.mobility_layout()
    if layout[3] > 0:
        # symmetric FP64 product: each unordered pair evaluated once and applied
        # both ways, 126 flop per unordered pair (FMA = 2, rsqrt = 1, counted
        # from pair_wall_sym and the pair's distances) against 2 x 119
        kname = "rpy_sym_f64<wall, tile %d>" % layout[3]
        executed = nb * (nb + 1) / 2 * SYM_WALL_FLOP_PER_UNORDERED_PAIR / avg_launch_s
    else:
        kname = "rpy_items_%s<wall>" % ("f64" if args.precision == "fp64" else "mixed")
        executed = achieved
    peak = fp64_peak if args.precision == "fp64" else fp32_peak
    clocks = clk.summary()
    roofline = {"bound": "alu", "achieved": achieved / 1e12,
                "peak": peak / 1e12, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": TRAFFIC_BYTES.get((args.precision, layout[3])),
                "kernel": kname, "layout": list(layout),
                "executed_tflops": executed / 1e12, "executed_frac": executed / peak,
                "algorithmic_vs_executed": "achieved counts N^2 pairs x 119 flop per launch; the symmetric "
                                           "kernel executes N(N+1)/2 x 126, so frac can exceed the FP64 "
                                           "pipe's busy fraction" if layout[3] > 0 else None,
                "flop_per_pair": fpp, "pairs_per_launch": nb * nb,
                "launch_ms": avg_launch_s * 1e3, "launches": mob_launches,
                "launch_timing": "CUDA events around each launch in %d further steps "
                                 "(host-launched Arnoldi steps)" % min(args.steps, 5),
                "peak_source": "measured %s FMA streams (am_alu_peak) on this GPU" %
                               ("DFMA" if args.precision == "fp64" else "FFMA"),
                "fp32_fma_peak_tflops": fp32_peak / 1e12, "fp64_fma_peak_tflops": fp64_peak / 1e12,
                "fp32_kernel": {"kernel": at_scale["mixed"]["kernel"], "blobs": at_scale["mixed"]["blobs"],
                                "launch_ms": at_scale["mixed"]["ms"], "frac": at_scale["mixed"]["frac_of_fma_peak"],
                                "achieved_tflops": at_scale["mixed"]["tflops"], "peak_tflops": fp32_peak / 1e12,
                                "peak_source": "measured FFMA streams (am_alu_peak) on this GPU",
                                "flop_per_pair": fpp},
                "fp32_kernel_symmetric": {"kernel": at_scale["mixed_symmetric"]["kernel"],
                                          "blobs": at_scale["mixed_symmetric"]["blobs"],
                                          "launch_ms": at_scale["mixed_symmetric"]["ms"],
                                          "frac": at_scale["mixed_symmetric"]["frac_of_fma_peak"],
                                          "note": "algorithmic count (N^2 x 119 flop); the kernel evaluates each "
                                                  "unordered pair once"}}
    cpu = None
    if world == 1:
        pool = OraclePool()
        rate, cp, nrows, el = oracle_sample(w, 0.0, pool, seconds=12.0)
        pool.close()
        cpu = {"value": rate, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
               "sample": "oracle mobility rows: %d of %d target blobs x %d sources, split over %d "
                         "worker processes (%.1f s)" % (nrows, nb, nb, pool.procs, el)}
    h2d = 6 * 3 * P * 8
    d2h = (6 * M + 3 * P + 3 * nb) * 8
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_s_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32-pairs/f64-sums",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "blobs": nb, "bodies": M, "links": P, "unknowns": n,
                       "precision": args.precision, "tol": TOL,
                       "l2": "512 MB buffer written between timed steps (inputs smaller than L2)",
                       "gmres": "device-resident cycles (CUDA graph WHILE node over Arnoldi steps)",
                       "parallelism": "independent suspension per GPU" if world > 1 else "1 GPU"},
            "solve_ms_per_step": 1e3 * total_s_all / args.steps,
            "gmres_iterations_per_step": statistics.mean(iters),
            "precond_build_ms_per_step": statistics.mean(precond_ms),
            "max_rel_residual": max(resid),
            "wall_s_timed_region": t_wall,
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_rate, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches), "clocks": clocks,
            "rk2_form": rk2_res, "guess_form": guess_res, "steric": steric, "single_blob_form": sb_res,
            "products_compared": compared, "matvec_at_scale": at_scale, "chains_solve": chains_res,
            "learned_form": learned_res, "batched_form": batched, "periodic_form": periodic_res,
            "bacteria_step": bact_res}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
