"""Oracle-S: the block-sparse FP64 oracle for windows whose dense system does not fit.

TEST INFRASTRUCTURE ONLY (like oracle/ba.py): only tests/, __graft_entry__.smoke() and
bench.py's CPU legs may use it.  It shares no code with the CUDA library.

The LM iteration is the dense oracle's, step for step (cuVSLAM Sec. 2.2, Eq. r^repr and
the SBA objective; Huber IRLS weights, Marquardt diagonal, Nielsen's damping update,
accept iff L > 0 and gain > 0, left SE(3) and Euclidean updates): `lm_iteration` below
calls oracle/ba.py's `apply_step`, `accept_step` and `nielsen_update`.  Only the linear
algebra differs: the normal equations are accumulated into their nonzero blocks and
factored by a generic block-sparse Cholesky (oracle/ba_sparse.c, built by
oracle/build.py), so windows with hundreds of thousands of landmarks fit in memory.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import ba
from .build import LIB, build

_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(LIB)
        vp, i, d, i64p = C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_int64)
        lib.bs_create.restype = vp
        lib.bs_create.argtypes = [i, i, i, i, i, vp, vp, vp, vp, vp, vp, i]
        lib.bs_destroy.restype = None
        lib.bs_destroy.argtypes = [vp]
        lib.bs_info.restype = None
        lib.bs_info.argtypes = [vp, i64p]
        lib.bs_evaluate.restype = None
        lib.bs_evaluate.argtypes = [vp, vp, vp, d, d, vp]
        lib.bs_linearise_solve.restype = i
        lib.bs_linearise_solve.argtypes = [vp, vp, vp, d, d, d, vp, vp, vp, vp]
        lib.bs_solve_rhs.restype = None
        lib.bs_solve_rhs.argtypes = [vp, vp, vp]
        lib.bs_pattern.restype = None
        lib.bs_pattern.argtypes = [vp, vp, vp]
        _lib = lib
    return _lib


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _p(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


class SparseWindow:
    """A window analysed once (observation grouping, block pattern of H and of its factor);
    linearise-and-solve and evaluate at any state."""

    def __init__(self, win: ba.Window, threads: int | None = None):
        lib = _load()
        self.win = win
        self.threads = default_threads() if threads is None else int(threads)
        # keep the arrays the C side borrows alive and contiguous
        self._intr = np.ascontiguousarray(win.intr, np.float64)
        self._tcb = np.ascontiguousarray(win.T_cb, np.float64).reshape(-1, 12)
        self._kf = np.ascontiguousarray(win.obs_kf, np.int32)
        self._cam = np.ascontiguousarray(win.obs_cam, np.int32)
        self._lm = np.ascontiguousarray(win.obs_lm, np.int32)
        self._uv = np.ascontiguousarray(win.obs_uv, np.float64)
        h = lib.bs_create(win.K, self._intr.shape[0], win.M, self._kf.size, win.fixed_kf, _p(self._intr),
                          _p(self._tcb), _p(self._kf), _p(self._cam), _p(self._lm), _p(self._uv), self.threads)
        if not h:
            raise ValueError("bs_create failed (bad sizes or indices, or out of memory)")
        self._h = C.c_void_p(h)
        info = np.zeros(6, np.int64)
        lib.bs_info(self._h, info.ctypes.data_as(C.POINTER(C.c_int64)))
        self.n_c, self.n_f, self.n_blocks, self.n_factor_blocks, self.n_factor_values, self.n_indep = map(int, info)

    def close(self):
        if getattr(self, "_h", None):
            _load().bs_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def evaluate(self, poses, lms) -> ba.Eval:
        """F, n_valid, n_inlier and RMS at (poses, lms), as oracle/ba.py's evaluate."""
        poses = np.ascontiguousarray(poses, np.float64)
        lms = np.ascontiguousarray(lms, np.float64)
        ev = np.zeros(4)
        _load().bs_evaluate(self._h, _p(poses), _p(lms), self.win.huber_delta, self.win.z_min, _p(ev))
        nv = int(ev[2])
        return ba.Eval(float(ev[0]), nv, int(ev[3]), math.sqrt(ev[1] / nv) if nv else 0.0)

    def linearise_solve(self, poses, lms, lam: float):
        """(delta or None if not positive definite, D, g, Eval at x) for (H + lam D) delta = -g,
        columns ordered as the dense oracle's: free keyframe twists, then landmarks."""
        poses = np.ascontiguousarray(poses, np.float64)
        lms = np.ascontiguousarray(lms, np.float64)
        delta, g, D = np.zeros(self.n_f), np.zeros(self.n_f), np.zeros(self.n_f)
        ev = np.zeros(4)
        ok = _load().bs_linearise_solve(self._h, _p(poses), _p(lms), float(lam), self.win.huber_delta,
                                        self.win.z_min, _p(delta), _p(g), _p(D), _p(ev))
        nv = int(ev[2])
        e = ba.Eval(float(ev[0]), nv, int(ev[3]), math.sqrt(ev[1] / nv) if nv else 0.0)
        return (delta if ok else None), D, g, e


    def solve_rhs(self, b) -> np.ndarray:
        """(H + lam D)^-1 b with the factor of the last successful linearise_solve."""
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros(self.n_f)
        _load().bs_solve_rhs(self._h, _p(b), _p(x))
        return x

    def pattern(self):
        """The factor's block pattern below the diagonal: (column pointers, block rows), block
        columns ordered landmarks first, then free keyframes."""
        cp = np.zeros(self.n_blocks + 1, np.int64)
        rows = np.zeros(max(self.n_factor_blocks, 1), np.int32)
        _load().bs_pattern(self._h, _p(cp), _p(rows))
        return cp, rows[:self.n_factor_blocks]


def lm_iteration(sw: SparseWindow, poses, lms, lam, nu):
    """One LM iteration, the dense oracle's steps with the sparse linear algebra.
    Returns (poses', lms', lam', nu', record)."""
    win = sw.win
    delta, D, g, ev = sw.linearise_solve(poses, lms, lam)
    if delta is None:
        rec = ba.IterRecord(ev.F, float("nan"), lam, float("nan"), float("nan"), float("nan"), False,
                            ev.n_valid, ev.n_inlier, ev.rms, True, None)
        lam_new, nu_new = ba.nielsen_update(lam, nu, float("nan"), False)
        return poses, lms, lam_new, nu_new, rec
    L = 0.5 * float(delta @ (lam * D * delta - g))
    p1, l1 = ba.apply_step(win, poses, lms, delta)
    F1 = sw.evaluate(p1, l1).F
    gain = (ev.F - F1) / L if L != 0.0 else float("nan")
    acc = ba.accept_step(L, F1, gain)
    rec = ba.IterRecord(ev.F, F1, lam, gain, L, float(np.linalg.norm(delta)), acc,
                        ev.n_valid, ev.n_inlier, ev.rms, False, delta)
    lam_new, nu_new = ba.nielsen_update(lam, nu, gain, acc)
    if acc:
        return p1, l1, lam_new, nu_new, rec
    return poses, lms, lam_new, nu_new, rec


def lm_solve(win: ba.Window, poses0, lms0, iters: int, lam0: float = 1e-4, keep_delta: bool = True,
             threads: int | None = None, sw: SparseWindow | None = None):
    """Exactly `iters` LM iterations; returns final (poses, lms, lam, nu) and the trace."""
    own = sw is None
    sw = SparseWindow(win, threads) if own else sw
    poses, lms, lam, nu = np.array(poses0, np.float64), np.array(lms0, np.float64), lam0, 2.0
    trace = []
    try:
        for _ in range(iters):
            poses, lms, lam, nu, rec = lm_iteration(sw, poses, lms, lam, nu)
            if not keep_delta:
                rec.delta = None
            trace.append(rec)
    finally:
        if own:
            sw.close()
    return poses, lms, lam, nu, trace
