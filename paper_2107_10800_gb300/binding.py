"""ctypes binding of libam.so (include/am.h).  Argument marshalling only:
every step of the solve runs in the library's CUDA kernels.  There is no CPU
fallback: if the library is missing or no GPU is present, calls raise.
"""
import ctypes
import os

import numpy as np

AM_OK = 0
AM_ERR_ARG = -1
AM_ERR_CUDA = -2
AM_ERR_NOT_CONVERGED = -3
AM_ERR_WALL_PENETRATION = -4
AM_ERR_NONUNIT_QUAT = -5
AM_ERR_SINGULAR = -6
AM_FP64 = 0
AM_MIXED = 1
AM_DF64 = 2

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libam.so")

# Every function the header declares, with its ctypes signature.
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p
_fp = ctypes.POINTER(ctypes.c_float)


class Config(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("blob_radius", ctypes.c_double),
                ("wall", ctypes.c_int), ("precision", ctypes.c_int),
                ("n_systems", ctypes.c_int), ("tol", ctypes.c_double),
                ("restart", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("corr_tol", ctypes.c_double), ("corr_max_iter", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p), ("single_blob", ctypes.c_int),
                ("box", ctypes.c_double * 3), ("ewald_tol", ctypes.c_double),
                ("ewald_xi", ctypes.c_double)]


class StepStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int),
                ("restarts", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("constraint_residual", ctypes.c_double),
                ("g2_before", ctypes.c_double), ("g2_after", ctypes.c_double),
                ("corr_iterations", ctypes.c_int), ("pairs", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_int), ("ms_precond", ctypes.c_double),
                ("ms_gmres", ctypes.c_double), ("ms_update", ctypes.c_double),
                ("learned_systems", ctypes.c_int), ("rel_residual0", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


SIGNATURES = {
    "am_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(_vp)]),
    "am_set_bodies": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _dp, _dp, _ip, _dp, _dp, _dp, _ip]),
    "am_set_constraints": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _ip, _ip, _dp, _dp, _dp, _dp]),
    "am_set_joints": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _ip, _ip, _dp]),
    "am_solve": (ctypes.c_int, [_vp, ctypes.POINTER(StepStats), _dp, _dp, _dp]),
    "am_solve_step": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, _dp, _dp,
                                     ctypes.POINTER(StepStats), _dp, _dp, _dp]),
    "am_solve_step_rk2": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, _dp, _dp, _dp,
                                         ctypes.POINTER(StepStats), _dp, _dp, _dp]),
    "am_get_bodies": (ctypes.c_int, [_vp, ctypes.c_int, _dp, _dp]),
    "am_get_blobs": (ctypes.c_int, [_vp, ctypes.c_int, _dp]),
    "am_apply_mobility": (ctypes.c_int, [_vp, _dp, _dp]),
    "am_apply_mobility_ex": (ctypes.c_int, [_vp, _dp, _dp, ctypes.c_int]),
    "am_set_mobility_layout": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "am_get_mobility_layout": (ctypes.c_int, [_vp, _ip]),
    "am_set_repulsion": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double]),
    "am_steric_forces": (ctypes.c_int, [_vp, _dp]),
    "am_apply_operator": (ctypes.c_int, [_vp, _dp, _dp]),
    "am_apply_precond": (ctypes.c_int, [_vp, _dp, _dp]),
    "am_rpy_matvec": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_int, _vp,
                                     ctypes.c_size_t, _vp]),
    "am_rpy_matvec_workspace": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int]),
    "am_rpy_matvec_rows": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, _vp,
                                          ctypes.c_size_t, _vp]),
    "am_rpy_matvec_rows_workspace": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "am_rpy_matvec_noalloc": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, ctypes.c_int, _vp]),
    "am_flops_per_pair": (ctypes.c_int, [ctypes.c_int]),
    "am_kernel_launches": (ctypes.c_longlong, []),
    "am_mobility_timing": (ctypes.c_int, [_vp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_longlong)]),
    "am_alu_peak": (ctypes.c_int, [ctypes.c_int, _dp]),
    "am_mlp_create": (ctypes.c_int, [ctypes.c_ulonglong, _vp, ctypes.POINTER(_vp)]),
    "am_mlp_destroy": (None, [_vp]),
    "am_mlp_num_params": (ctypes.c_int, []),
    "am_mlp_get_params": (ctypes.c_int, [_vp, _fp]),
    "am_mlp_set_params": (ctypes.c_int, [_vp, _fp]),
    "am_mlp_set_norm": (ctypes.c_int, [_vp, _fp, _fp, _fp]),
    "am_mlp_loss_grad": (ctypes.c_int, [_vp, _fp, _fp, ctypes.c_int, _dp, _fp]),
    "am_mlp_train": (ctypes.c_int, [_vp, _fp, _fp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_ulonglong, _dp]),
    "am_mlp_predict": (ctypes.c_int, [_vp, _fp, ctypes.c_int, ctypes.c_int, _fp]),
    "am_learned_features": (ctypes.c_int, [_vp, _fp, _fp]),
    "am_set_learned": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "am_set_initial_guess": (ctypes.c_int, [_vp, ctypes.c_int]),
    "am_periodic_info": (ctypes.c_int, [_vp, _dp, ctypes.POINTER(ctypes.c_longlong)]),
    "am_destroy": (None, [_vp]),
    "am_last_error": (ctypes.c_char_p, [_vp]),
}

_LIB = None


def lib():
    """Load libam.so once; raise if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libam.so is not built (call paper_2107_10800_gb300.build.build()); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


class AmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libam error %d: %s" % (code, msg))
        self.code = code


def _d(a, n=None):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=np.float64).ravel()
    if n is not None and arr.size != n:
        raise ValueError("expected %d values, got %d" % (n, arr.size))
    return arr, arr.ctypes.data_as(_dp)


def _i(a):
    arr = np.ascontiguousarray(a, dtype=np.int32).ravel()
    return arr, arr.ctypes.data_as(_ip)


def _out(n):
    arr = np.empty(n, dtype=np.float64)
    return arr, arr.ctypes.data_as(_dp)


class Solver:
    """One handle of the library (am_create ... am_destroy)."""

    def __init__(self, eta=1.0, a=0.1, wall=0, precision="fp64", tol=1e-10, restart=50,
                 max_iter=500, corr_tol=1e-10, corr_max_iter=20, stream=None, n_systems=1,
                 single_blob=False, box=None, ewald_tol=0.0, ewald_xi=0.0):
        """box: (Lx, Ly, Lz) of a triply periodic box, or None (unbounded)."""
        L = lib()
        prec = {"fp64": AM_FP64, "mixed": AM_MIXED}[precision]
        bx = (ctypes.c_double * 3)(*([0.0, 0.0, 0.0] if box is None else [float(v) for v in box]))
        cfg = Config(eta, a, wall, prec, n_systems, tol, restart, max_iter, corr_tol, corr_max_iter,
                     stream, 1 if single_blob else 0, bx, ewald_tol, ewald_xi)
        self.single_blob = bool(single_blob)
        h = _vp()
        rc = L.am_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != AM_OK:
            raise AmError(rc, "am_create failed (" + L.am_last_error(None).decode() + ")")
        self.h = h
        self.S = n_systems
        self.sizes = [(0, 0, 0)] * n_systems  # (bodies, blobs, links) per system

    @property
    def M(self):
        return sum(z[0] for z in self.sizes)

    @property
    def Nb(self):
        return sum(z[1] for z in self.sizes)

    @property
    def P(self):
        return sum(z[2] for z in self.sizes)

    def _check(self, rc, allow_nc=False):
        if rc == AM_OK or (allow_nc and rc == AM_ERR_NOT_CONVERGED):
            return rc
        raise AmError(rc, lib().am_last_error(self.h).decode())

    def close(self):
        if self.h:
            lib().am_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_bodies(self, q, theta, blob_offset, rho, F, assembly, slip=None, system=0):
        M = len(np.asarray(theta).reshape(-1, 4))
        if self.single_blob:  # the body is the blob: no blob arrays
            blob_offset, rho, slip = np.zeros(M + 1, np.int32), np.zeros((1, 3)), None
        off, off_p = _i(blob_offset)
        Nb = int(off[-1])
        qa, qp = _d(q, 3 * M)
        ta, tp = _d(theta, 4 * M)
        ra, rp = _d(rho, 3 * Nb if not self.single_blob else 3)
        fa, fp = _d(F, 6 * M)
        sa, sp = _d(slip, 3 * Nb)
        aa, ap = _i(assembly)
        self._check(lib().am_set_bodies(self.h, system, M, qp, tp, off_p, rp, fp, sp, ap))
        self.sizes = list(self.sizes)
        self.sizes[system] = (M, Nb, 0)

    def set_constraints(self, body_p, body_q, dl_p, dl_q, dl_p_dot=None, dl_q_dot=None, system=0):
        bp, bpp = _i(body_p)
        bq, bqp = _i(body_q)
        P = len(bp)
        a1, p1 = _d(dl_p, 3 * P)
        a2, p2 = _d(dl_q, 3 * P)
        a3, p3 = _d(dl_p_dot, 3 * P)
        a4, p4 = _d(dl_q_dot, 3 * P)
        self._check(lib().am_set_constraints(self.h, system, P, bpp, bqp, p1, p2, p3, p4))
        self.sizes = list(self.sizes)
        self.sizes[system] = (self.sizes[system][0], self.sizes[system][1], P)

    def set_joints(self, body_p, body_q, joints, system=0):
        bp, bpp = _i(body_p)
        bq, bqp = _i(body_q)
        P = len(bp)
        ja, jp = _d(joints, 3 * P)
        self._check(lib().am_set_joints(self.h, system, P, bpp, bqp, jp))
        self.sizes = list(self.sizes)
        self.sizes[system] = (self.sizes[system][0], self.sizes[system][1], P)

    @property
    def n(self):
        return 3 * self.Nb + 6 * self.M + 3 * self.P

    def solve(self):
        st = StepStats()
        U, Up = _out(6 * self.M)
        phi, pp = _out(3 * self.P)
        lam, lp = _out(3 * self.Nb)
        self._check(lib().am_solve(self.h, ctypes.byref(st), Up, pp, lp), allow_nc=True)
        return U.reshape(-1, 6), phi.reshape(-1, 3), lam.reshape(-1, 3), st.as_dict()

    def step(self, t, dt, dl_next=None):
        st = StepStats()
        U, Up = _out(6 * self.M)
        phi, pp = _out(3 * self.P)
        lam, lp = _out(3 * self.Nb)
        if dl_next is None:
            a1 = a2 = None
            p1 = p2 = None
        else:
            a1, p1 = _d(dl_next[0], 3 * self.P)
            a2, p2 = _d(dl_next[1], 3 * self.P)
        self._check(lib().am_solve_step(self.h, t, dt, p1, p2, ctypes.byref(st), Up, pp, lp),
                    allow_nc=True)
        return U.reshape(-1, 6), phi.reshape(-1, 3), lam.reshape(-1, 3), st.as_dict()

    def step_rk2(self, t, dt, dl_half=None, dl_next=None):
        """Explicit midpoint step; dl_half = (dlp, dlq) or (dlp, dlq, dlpd,
        dlqd) at t + dt/2, dl_next = (dlp, dlq) at t + dt (None: keep)."""
        st = StepStats()
        U, Up = _out(6 * self.M)
        phi, pp = _out(3 * self.P)
        lam, lp = _out(3 * self.Nb)
        keep = []

        def arr(v):
            if v is None:
                return None
            a, p = _d(v, 3 * self.P)
            keep.append(a)
            return p
        h = list(dl_half) if dl_half is not None else [None, None]
        h += [None] * (4 - len(h))
        nx = list(dl_next) if dl_next is not None else [None, None]
        self._check(lib().am_solve_step_rk2(self.h, t, dt, arr(h[0]), arr(h[1]), arr(h[2]), arr(h[3]),
                                            arr(nx[0]), arr(nx[1]), ctypes.byref(st), Up, pp, lp),
                    allow_nc=True)
        return U.reshape(-1, 6), phi.reshape(-1, 3), lam.reshape(-1, 3), st.as_dict()

    def bodies(self, system=0):
        M = self.sizes[system][0]
        q, qp = _out(3 * M)
        th, tp = _out(4 * M)
        self._check(lib().am_get_bodies(self.h, system, qp, tp))
        return q.reshape(-1, 3), th.reshape(-1, 4)

    def blobs(self, system=0):
        Nb = self.sizes[system][1]
        r, rp = _out(3 * Nb)
        self._check(lib().am_get_blobs(self.h, system, rp))
        return r.reshape(-1, 3)

    def split(self, U, phi, lam):
        """Per-system views of solve outputs (which concatenate the systems)."""
        out, b0, l0, p0 = [], 0, 0, 0
        for M, Nb, P in self.sizes:
            out.append((U[b0:b0 + M], phi[p0:p0 + P], lam[l0:l0 + Nb]))
            b0 += M; l0 += Nb; p0 += P
        return out

    def apply_mobility(self, lam):
        """u = M lambda (3Nb); with single_blob the body mobility, (f, tau)
        per body in and (u, omega) out (6M)."""
        k = 6 * self.M if self.single_blob else 3 * self.Nb
        la, lp = _d(lam, k)
        u, up = _out(k)
        self._check(lib().am_apply_mobility(self.h, lp, up))
        return u.reshape(-1, 6 if self.single_blob else 3)

    def apply_mobility_ex(self, lam, arithmetic):
        """u = M lambda with the pair arithmetic "fp64", "mixed" or "df64"."""
        mode = {"fp64": AM_FP64, "mixed": AM_MIXED, "df64": AM_DF64}[arithmetic]
        la, lp = _d(lam, 3 * self.Nb)
        u, up = _out(3 * self.Nb)
        self._check(lib().am_apply_mobility_ex(self.h, lp, up, mode))
        return u.reshape(-1, 3)

    def periodic_info(self):
        """Parameters of a periodic handle's product (am_periodic_info)."""
        d = np.empty(6, np.float64)
        i = np.empty(6, np.int64)
        self._check(lib().am_periodic_info(self.h, d.ctypes.data_as(_dp),
                                           i.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))))
        return {"xi": d[0], "r_c": d[1], "beta": d[2], "h": tuple(d[3:6]),
                "grid": tuple(int(v) for v in i[0:3]), "support": int(i[3]),
                "real_pairs": int(i[4]), "cells": int(i[5])}

    def mobility_layout(self):
        """(targets per thread, source chunk, targets per item, symmetric
        tile or 0) of the all-pairs product in use (am_get_mobility_layout)."""
        a = np.zeros(4, np.int32)
        self._check(lib().am_get_mobility_layout(self.h, a.ctypes.data_as(_ip)))
        return tuple(int(v) for v in a)

    def set_repulsion(self, eps, range_, cutoff, eps_wall=0.0, range_wall=1.0):
        """Steric repulsion between articulated bodies and with the wall."""
        self._check(lib().am_set_repulsion(self.h, eps, range_, cutoff, eps_wall, range_wall))

    def steric_forces(self):
        f, fp = _out(3 * self.Nb)
        self._check(lib().am_steric_forces(self.h, fp))
        return f.reshape(-1, 3)

    def set_initial_guess(self, order):
        """Initial guess of the time-step solves: 0 P~^-1 b, 1 the previous
        solution, 2 or 3 the extrapolation in time through the last 2 or 3."""
        self._check(lib().am_set_initial_guess(self.h, int(order)))

    def set_mobility_layout(self, targets_per_thread, source_chunk=0):
        """Fix the all-pairs product layout (0 targets per thread: autotune)."""
        self._check(lib().am_set_mobility_layout(self.h, targets_per_thread, source_chunk))

    def apply_operator(self, y):
        ya, yp = _d(y, self.n)
        o, op = _out(self.n)
        self._check(lib().am_apply_operator(self.h, yp, op))
        return o

    def apply_precond(self, r):
        ra, rp = _d(r, self.n)
        o, op = _out(self.n)
        self._check(lib().am_apply_precond(self.h, rp, op))
        return o

    def learned_features(self, targets=False):
        """Features (M x 144) of all bodies at the current pose and, with
        targets=True, the background-flow targets (M x 32) of the last
        solve's solution."""
        X = np.empty((self.M, MLP_FEAT), dtype=np.float32)
        T = np.empty((self.M, MLP_OUT), dtype=np.float32) if targets else None
        rc = lib().am_learned_features(self.h, X.ctypes.data_as(_fp),
                                       T.ctypes.data_as(_fp) if targets else None)
        self._check(rc)
        return (X, T) if targets else X

    def set_learned(self, model, check=True):
        """Use `model` (an Mlp, or None) for the initial guess of cold starts."""
        self._mlp = model  # keep it alive while the handle uses it
        rc = lib().am_set_learned(self.h, model.m if model is not None else None, 1 if check else 0)
        self._check(rc)

    def mobility_timing(self, enable):
        """(total ms, launches) of the all-pairs kernel recorded so far;
        enable=True clears and starts recording, False stops."""
        ms = ctypes.c_double()
        k = ctypes.c_longlong()
        self._check(lib().am_mobility_timing(self.h, 1 if enable else 0, ctypes.byref(ms),
                                             ctypes.byref(k)))
        return ms.value, k.value

    def load(self, w, system=0, t=0.0):
        """Set system `system` from a workload dict of
        paper_2107_10800_gb300.workloads."""
        self.set_bodies(w["q"], w["theta"], w["blob_offset"], w["rho"], w["F"], w["assembly"],
                        system=system)
        if len(w["body_p"]):
            if w.get("dl") is not None:
                dlp, dlq, dlpd, dlqd = w["dl"](t)
                self.set_constraints(w["body_p"], w["body_q"], dlp, dlq, dlpd, dlqd, system=system)
            else:
                self.set_joints(w["body_p"], w["body_q"], w["joints"], system=system)

    @classmethod
    def from_workload(cls, w, t=0.0, **kw):
        """A solver holding one workload dict (a periodic one when the dict
        has a "box")."""
        if w.get("box") is not None and "box" not in kw:
            kw["box"] = w["box"]
        s = cls(eta=w["eta"], a=w["a"], wall=w["wall"], **kw)
        s.load(w, 0, t)
        return s

    @classmethod
    def from_workloads(cls, ws, t=0.0, **kw):
        """A solver holding several independent workloads (one system each;
        they must share eta, a and wall)."""
        w0 = ws[0]
        s = cls(eta=w0["eta"], a=w0["a"], wall=w0["wall"], n_systems=len(ws), **kw)
        for k, w in enumerate(ws):
            s.load(w, k, t)
        return s


MLP_FEAT = 144
MLP_OUT = 32


def _f32(a, shape=None):
    arr = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None and arr.shape != shape:
        arr = arr.reshape(shape)
    return arr, arr.ctypes.data_as(_fp)


class Mlp:
    """The learned initial-guess network of the library (am_mlp_*)."""

    def __init__(self, seed=0, stream=None):
        m = _vp()
        rc = lib().am_mlp_create(seed, stream, ctypes.byref(m))
        if rc != AM_OK:
            raise AmError(rc, lib().am_last_error(None).decode())
        self.m = m
        self.n_params = int(lib().am_mlp_num_params())

    def _check(self, rc):
        if rc != AM_OK:
            raise AmError(rc, lib().am_last_error(None).decode())

    def close(self):
        if self.m:
            lib().am_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        p = np.empty(self.n_params, dtype=np.float32)
        self._check(lib().am_mlp_get_params(self.m, p.ctypes.data_as(_fp)))
        return p

    def set_params(self, p):
        arr, ptr = _f32(np.ravel(p))
        if arr.size != self.n_params:
            raise ValueError("expected %d parameters" % self.n_params)
        self._check(lib().am_mlp_set_params(self.m, ptr))

    def set_norm(self, mu, sd, sd_out):
        a, pa = _f32(np.ravel(mu))
        b, pb = _f32(np.ravel(sd))
        c, pc = _f32(np.ravel(sd_out))
        if a.size != MLP_FEAT or b.size != MLP_FEAT or c.size != MLP_OUT:
            raise ValueError("mu, sd: 144 values; sd_out: 32")
        self._check(lib().am_mlp_set_norm(self.m, pa, pb, pc))

    def loss_grad(self, X, T):
        x, px = _f32(X)
        t, pt = _f32(T)
        n = x.shape[0]
        if x.shape != (n, MLP_FEAT) or t.shape != (n, MLP_OUT):
            raise ValueError("X: n x 144, T: n x 32")
        loss = ctypes.c_double()
        g = np.empty(self.n_params, dtype=np.float32)
        self._check(lib().am_mlp_loss_grad(self.m, px, pt, n, ctypes.byref(loss), g.ctypes.data_as(_fp)))
        return loss.value, g

    def train(self, X, T, epochs, batch=256, lr=1e-3, seed=0):
        x, px = _f32(X)
        t, pt = _f32(T)
        n = x.shape[0]
        if x.shape != (n, MLP_FEAT) or t.shape != (n, MLP_OUT):
            raise ValueError("X: n x 144, T: n x 32")
        loss = ctypes.c_double()
        self._check(lib().am_mlp_train(self.m, px, pt, n, epochs, batch, lr, seed, ctypes.byref(loss)))
        return loss.value

    def predict(self, X, bf16=True):
        x, px = _f32(X)
        n = x.shape[0]
        if x.shape != (n, MLP_FEAT):
            raise ValueError("X: n x 144")
        Y = np.empty((n, MLP_OUT), dtype=np.float32)
        self._check(lib().am_mlp_predict(self.m, px, n, 1 if bf16 else 0, Y.ctypes.data_as(_fp)))
        return Y


def rpy_matvec_ptr(d_r, d_lam, d_u, n, eta, a, wall, precision, d_work, work_bytes, stream=None):
    """am_rpy_matvec on raw device pointers (ints)."""
    prec = {"fp64": AM_FP64, "mixed": AM_MIXED}.get(precision, precision)
    rc = lib().am_rpy_matvec(d_r, d_lam, d_u, n, eta, a, wall, prec, d_work, work_bytes, stream)
    if rc != AM_OK:
        raise AmError(rc, lib().am_last_error(None).decode())


def rpy_matvec_noalloc_ptr(d_r, d_lam, d_u, n, eta, a, wall, precision, stream=None):
    """am_rpy_matvec_noalloc on raw device pointers (ints): the mobility
    product with the library's fixed scratch array instead of a workspace,
    for callers that cannot allocate device memory."""
    prec = {"fp64": AM_FP64, "mixed": AM_MIXED}.get(precision, precision)
    rc = lib().am_rpy_matvec_noalloc(d_r, d_lam, d_u, n, eta, a, wall, prec, stream)
    if rc != AM_OK:
        raise AmError(rc, lib().am_last_error(None).decode())


NOALLOC_SCRATCH_BYTES = 8 << 20


def rpy_matvec_rows_ptr(d_r, d_lam, d_u, n, row0, nrows, eta, a, wall, precision, d_work, work_bytes,
                        stream=None):
    """am_rpy_matvec_rows on raw device pointers (ints)."""
    prec = {"fp64": AM_FP64, "mixed": AM_MIXED}.get(precision, precision)
    rc = lib().am_rpy_matvec_rows(d_r, d_lam, d_u, n, row0, nrows, eta, a, wall, prec, d_work, work_bytes,
                                  stream)
    if rc != AM_OK:
        raise AmError(rc, lib().am_last_error(None).decode())


def rpy_matvec_rows_workspace(n, nrows, precision):
    prec = {"fp64": AM_FP64, "mixed": AM_MIXED}.get(precision, precision)
    return int(lib().am_rpy_matvec_rows_workspace(n, nrows, prec))


def rpy_matvec_workspace(n, precision):
    prec = {"fp64": AM_FP64, "mixed": AM_MIXED}.get(precision, precision)
    return int(lib().am_rpy_matvec_workspace(n, prec))


def flops_per_pair(wall):
    return int(lib().am_flops_per_pair(wall))


def alu_peak(fp64):
    """Measured FMA throughput (FLOP/s) of the current device."""
    f = ctypes.c_double()
    rc = lib().am_alu_peak(1 if fp64 else 0, ctypes.byref(f))
    if rc != AM_OK:
        raise AmError(rc, "am_alu_peak failed")
    return f.value


def kernel_launches():
    return int(lib().am_kernel_launches())
