"""Thin ctypes binding of the C ABI in include/cvba.h (argument marshalling only).

Every step of the solve runs in the CUDA library libcvba.so; this module only converts
numpy arrays to pointers and status codes to exceptions.  If the library has not been
built, importing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcvba.so")

CVBA_FP64 = 0
CVBA_MIXED = 1
STATUS = {0: "CVBA_OK", 1: "CVBA_ERR_INVALID_ARG", 2: "CVBA_ERR_INDEX", 3: "CVBA_ERR_NONFINITE",
          4: "CVBA_ERR_CUDA", 5: "CVBA_ERR_OOM", 6: "CVBA_ERR_NOT_PD", 7: "CVBA_ERR_TIMEOUT",
          8: "CVBA_ERR_STATE"}


class cvba_opts(C.Structure):
    _fields_ = [("iters", C.c_int), ("huber_delta", C.c_double), ("lambda0", C.c_double),
                ("z_min", C.c_double), ("reset_lambda", C.c_int), ("refine", C.c_int)]


class cvba_iter(C.Structure):
    _fields_ = [("cost0", C.c_double), ("cost1", C.c_double), ("lambda_", C.c_double),
                ("gain", C.c_double), ("pred", C.c_double), ("step_norm", C.c_double),
                ("rms_px", C.c_double), ("accepted", C.c_int), ("nonpd", C.c_int),
                ("n_valid", C.c_int), ("n_inlier", C.c_int), ("berr", C.c_double), ("refined", C.c_int),
                ("reserved", C.c_int)]


def make_opts(iters, huber_delta=1.0, lambda0=1e-4, z_min=1e-3, reset_lambda=True, refine=-1) -> "cvba_opts":
    """cvba_opts; refine < 0 selects the precision's default (1 for mixed, 0 for FP64)."""
    return cvba_opts(int(iters), float(huber_delta), float(lambda0), float(z_min), 1 if reset_lambda else 0,
                     int(refine))


ITER_DTYPE = np.dtype([("cost0", "f8"), ("cost1", "f8"), ("lambda", "f8"), ("gain", "f8"), ("pred", "f8"),
                       ("step_norm", "f8"), ("rms_px", "f8"), ("accepted", "i4"), ("nonpd", "i4"),
                       ("n_valid", "i4"), ("n_inlier", "i4"), ("berr", "f8"), ("refined", "i4"), ("reserved", "i4")])
assert ITER_DTYPE.itemsize == C.sizeof(cvba_iter)


LM_RECORD_DTYPE = np.dtype([("cost0", "f8"), ("cost1", "f8"), ("lambda", "f8"), ("gain", "f8"), ("pred", "f8"),
                           ("step_norm", "f8"), ("rms_px", "f8"), ("accepted", "i4"), ("nonpd", "i4"),
                           ("n_valid", "i4"), ("n_inlier", "i4"), ("n_bad_index", "i4"), ("reserved", "i4")])


class CvbaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
                          " (the CUDA library is required; there is no CPU path)")
    lib = C.CDLL(LIB_PATH)
    vp, i, d, dp, ip = C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_int32)
    sig = {
        "cvba_create": (i, [C.POINTER(vp), i, vp, i]),
        "cvba_destroy": (None, [vp]),
        "cvba_status_string": (C.c_char_p, [i]),
        "cvba_last_error": (C.c_char_p, [vp]),
        "cvba_set_rig": (i, [vp, i, dp, dp, ip]),
        "cvba_get_rig": (i, [vp, dp, dp, ip]),
        "cvba_get_state": (i, [vp, vp, C.POINTER(C.c_size_t)]),
        "cvba_set_state": (i, [vp, vp, C.c_size_t]),
        "cvba_set_poses": (i, [vp, i, dp, i]),
        "cvba_set_landmarks": (i, [vp, i, dp]),
        "cvba_set_observations": (i, [vp, i, ip, ip, ip, dp]),
        "cvba_solve": (i, [vp, C.POINTER(cvba_opts), vp]),
        "cvba_evaluate": (i, [vp, d, d, dp, dp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "cvba_get_poses": (i, [vp, dp]),
        "cvba_get_landmarks": (i, [vp, dp]),
        "cvba_get_increment": (i, [vp, dp]),
        "cvba_get_damping": (i, [vp, dp, dp]),
        "cvba_set_damping": (i, [vp, d, d]),
        "cvba_get_layout": (i, [vp, ip, ip, ip]),
        "cvba_get_sizes": (i, [vp] + [C.POINTER(C.c_int)] * 5),
        "cvba_solve_launch_count": (i, [vp, i, C.POINTER(C.c_int)]),
        "cvba_solve_async": (i, [vp, C.POINTER(cvba_opts)]),
        "cvba_get_trace": (i, [vp, vp, i]),
        "cvba_set_poses_dev": (i, [vp, vp]),
        "cvba_set_landmarks_dev": (i, [vp, vp]),
        "cvba_get_poses_dev": (i, [vp, vp]),
        "cvba_get_landmarks_dev": (i, [vp, vp]),
        "cvba_profile_iteration": (i, [vp, C.POINTER(cvba_opts), i, C.POINTER(C.c_float), C.POINTER(C.c_int)]),
        "cvba_profile_names": (C.c_char_p, []),
        "cvba_evaluate_noalloc": (i, [i, i, i, i] + [vp] * 8 + [d, d, vp, vp]),
        "cvba_pnp_solve": (i, [i, i, i, i, i] + [vp] * 8 + [C.POINTER(cvba_opts), vp, vp]),
        "cvba_pnp_kernels_per_solve": (i, []),
        "cvba_pgo_workspace_bytes": (C.c_size_t, [i, i]),
        "cvba_pgo_solve": (i, [i, i, vp, vp, vp, i, C.POINTER(cvba_opts), vp, vp, C.c_size_t, vp]),
        "cvba_relpose_solve": (i, [i, i, i, i, i] + [vp] * 9 + [C.POINTER(cvba_opts), vp, vp]),
        "cvba_triangulate": (i, [i, i, i, i, i] + [vp] * 7 + [C.POINTER(cvba_opts)] + [vp] * 5),
        "cvba_set_tuning": (i, [vp, i, i]),
        "cvba_set_chol_mode": (i, [vp, i]),
        "cvba_batch_create": (i, [C.POINTER(vp), i, C.POINTER(vp)]),
        "cvba_batch_destroy": (None, [vp]),
        "cvba_batch_last_error": (C.c_char_p, [vp]),
        "cvba_batch_solve": (i, [vp, C.POINTER(cvba_opts), vp]),
        "cvba_batch_solve_async": (i, [vp, C.POINTER(cvba_opts)]),
        "cvba_batch_launch_count": (i, [vp, C.POINTER(cvba_opts), C.POINTER(C.c_int)]),
        "cvba_batch_set_chol_cluster": (i, [vp, i]),
        "cvba_batch_autotune": (i, [vp, C.POINTER(cvba_opts)] + [C.POINTER(C.c_int)] * 3),
        "cvba_batch_autotune_clear": (None, []),
        "cvba_cost_workspace_bytes": (C.c_size_t, [i, i, i]),
        "cvba_cost_forward": (i, [i, i, i, i, i] + [vp] * 9 + [d, d, vp, vp, C.c_size_t, vp]),
        "cvba_cost_backward": (i, [i, i, i, i, i] + [vp] * 9 + [d, d, vp, vp, vp, vp, vp, vp, C.c_size_t, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


class Context:
    """One BA window on one GPU (owns a cvba_ctx)."""

    def __init__(self, precision: str | int = "fp64", device: int = 0, stream: int | None = None):
        prec = {"fp64": CVBA_FP64, "mixed": CVBA_MIXED}.get(precision, precision)
        h = C.c_void_p()
        st = lib.cvba_create(C.byref(h), int(device), C.c_void_p(stream) if stream else None, int(prec))
        if st != 0:
            raise CvbaError(st, "cvba_create failed (a GB300 / sm_103 device is required)")
        self._h = h
        self.precision = prec

    def close(self):
        if getattr(self, "_h", None):
            lib.cvba_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _check(self, st: int):
        if st != 0:
            raise CvbaError(st, lib.cvba_last_error(self._h).decode())

    # --- setters
    def cvba_set_rig(self, intr, T_cb, wh=None):
        intr, T_cb = _f64(intr).reshape(-1, 4), _f64(T_cb).reshape(-1, 12)
        whp = None
        if wh is not None:
            wh = _i32(wh).reshape(-1, 2)
            whp = _iptr(wh)
        self._check(lib.cvba_set_rig(self._h, intr.shape[0], _dptr(intr), _dptr(T_cb), whp))

    def cvba_get_rig(self):
        C_ = self.cvba_get_sizes()["C"]
        intr, T_cb, wh = np.zeros((C_, 4)), np.zeros((C_, 3, 4)), np.zeros((C_, 2), np.int32)
        self._check(lib.cvba_get_rig(self._h, _dptr(intr), _dptr(T_cb), _iptr(wh)))
        return intr, T_cb, wh

    def cvba_get_state(self) -> bytes:
        """Checkpoint of the solve state (poses, landmarks, damping) as bytes."""
        n = C.c_size_t()
        self._check(lib.cvba_get_state(self._h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(lib.cvba_get_state(self._h, buf, C.byref(n)))
        return buf.raw[:n.value]

    def cvba_set_state(self, state: bytes):
        buf = C.create_string_buffer(bytes(state), len(state))
        self._check(lib.cvba_set_state(self._h, buf, len(state)))

    def cvba_set_poses(self, T_bw, fixed_kf: int = 0):
        T = _f64(T_bw).reshape(-1, 12)
        self._check(lib.cvba_set_poses(self._h, T.shape[0], _dptr(T), int(fixed_kf)))

    def cvba_set_landmarks(self, p_w):
        p = _f64(p_w).reshape(-1, 3)
        self._check(lib.cvba_set_landmarks(self._h, p.shape[0], _dptr(p)))

    def cvba_set_observations(self, kf, cam, lm, uv):
        kf, cam, lm, uv = _i32(kf), _i32(cam), _i32(lm), _f64(uv).reshape(-1, 2)
        self._check(lib.cvba_set_observations(self._h, kf.size, _iptr(kf), _iptr(cam), _iptr(lm), _dptr(uv)))

    # --- solve
    def cvba_solve(self, iters: int, huber_delta: float = 1.0, lambda0: float = 1e-4, z_min: float = 1e-3,
                   reset_lambda: bool = True, refine: int = -1) -> np.ndarray:
        o = make_opts(iters, huber_delta, lambda0, z_min, reset_lambda, refine)
        trace = np.zeros(max(int(iters), 1), ITER_DTYPE)
        self._check(lib.cvba_solve(self._h, C.byref(o), C.c_void_p(trace.ctypes.data)))
        return trace[:int(iters)]

    def cvba_evaluate(self, huber_delta: float = 1.0, z_min: float = 1e-3):
        cost, rms = C.c_double(), C.c_double()
        nv, ni = C.c_int(), C.c_int()
        self._check(lib.cvba_evaluate(self._h, float(huber_delta), float(z_min), C.byref(cost), C.byref(rms),
                                      C.byref(nv), C.byref(ni)))
        return dict(cost=cost.value, rms=rms.value, n_valid=nv.value, n_inlier=ni.value)

    # --- getters
    def cvba_get_sizes(self):
        v = [C.c_int() for _ in range(5)]
        self._check(lib.cvba_get_sizes(self._h, *[C.byref(x) for x in v]))
        return dict(zip(["K", "C", "M", "N", "P"], [x.value for x in v]))

    def cvba_get_poses(self) -> np.ndarray:
        K = self.cvba_get_sizes()["K"]
        out = np.zeros((K, 3, 4))
        self._check(lib.cvba_get_poses(self._h, _dptr(out)))
        return out

    def cvba_get_landmarks(self) -> np.ndarray:
        M = self.cvba_get_sizes()["M"]
        out = np.zeros((M, 3))
        self._check(lib.cvba_get_landmarks(self._h, _dptr(out)))
        return out

    def cvba_get_increment(self) -> np.ndarray:
        s = self.cvba_get_sizes()
        out = np.zeros(6 * (s["K"] - 1) + 3 * s["M"])
        self._check(lib.cvba_get_increment(self._h, _dptr(out)))
        return out

    def cvba_get_damping(self):
        lam, nu = C.c_double(), C.c_double()
        self._check(lib.cvba_get_damping(self._h, C.byref(lam), C.byref(nu)))
        return lam.value, nu.value

    def cvba_set_damping(self, lam: float, nu: float):
        self._check(lib.cvba_set_damping(self._h, float(lam), float(nu)))

    def cvba_get_layout(self):
        s = self.cvba_get_sizes()
        lo = np.zeros(s["M"], np.int32)
        oo = np.zeros(s["N"], np.int32)
        off = np.zeros(s["M"] + 1, np.int32)
        self._check(lib.cvba_get_layout(self._h, _iptr(lo), _iptr(oo), _iptr(off)))
        return lo, oo, off

    def cvba_solve_launch_count(self, iters: int) -> int:
        n = C.c_int()
        self._check(lib.cvba_solve_launch_count(self._h, int(iters), C.byref(n)))
        return n.value

    # --- asynchronous / device-pointer calls (pointers are device addresses, e.g. a
    #     torch tensor's data_ptr())
    def cvba_solve_async(self, iters: int, huber_delta: float = 1.0, lambda0: float = 1e-4, z_min: float = 1e-3,
                         reset_lambda: bool = True, refine: int = -1):
        o = make_opts(iters, huber_delta, lambda0, z_min, reset_lambda, refine)
        self._check(lib.cvba_solve_async(self._h, C.byref(o)))

    def cvba_get_trace(self, n: int) -> np.ndarray:
        trace = np.zeros(max(int(n), 1), ITER_DTYPE)
        self._check(lib.cvba_get_trace(self._h, C.c_void_p(trace.ctypes.data), int(n)))
        return trace[:int(n)]

    def cvba_set_poses_dev(self, ptr: int):
        self._check(lib.cvba_set_poses_dev(self._h, C.c_void_p(ptr)))

    def cvba_set_landmarks_dev(self, ptr: int):
        self._check(lib.cvba_set_landmarks_dev(self._h, C.c_void_p(ptr)))

    def cvba_get_poses_dev(self, ptr: int):
        self._check(lib.cvba_get_poses_dev(self._h, C.c_void_p(ptr)))

    def cvba_get_landmarks_dev(self, ptr: int):
        self._check(lib.cvba_get_landmarks_dev(self._h, C.c_void_p(ptr)))

    def cvba_profile_iteration(self, reps: int, huber_delta: float = 1.0, lambda0: float = 1e-4,
                               z_min: float = 1e-3, refine: int = -1) -> dict:
        o = make_opts(reps, huber_delta, lambda0, z_min, True, refine)
        n = C.c_int()
        self._check(lib.cvba_profile_iteration(self._h, C.byref(o), int(reps), None, C.byref(n)))
        ms = (C.c_float * n.value)()
        self._check(lib.cvba_profile_iteration(self._h, C.byref(o), int(reps), ms, C.byref(n)))
        names = lib.cvba_profile_names().decode().split(",")
        return dict(zip(names, [float(x) for x in ms]))

    def cvba_set_tuning(self, lin_tile_pairs: int = 0, schur_tile_landmarks: int = 0):
        self._check(lib.cvba_set_tuning(self._h, int(lin_tile_pairs), int(schur_tile_landmarks)))

    def cvba_set_chol_mode(self, mode: int = 0):
        """0: by size, 1: cluster form, 2: blocked form of the reduced-system factorisation."""
        self._check(lib.cvba_set_chol_mode(self._h, int(mode)))

    # --- convenience
    def load(self, problem, poses=None, landmarks=None):
        """Load a synth.Problem (rig, initial poses and landmarks, observations)."""
        self.cvba_set_rig(problem.rig.intr, problem.rig.T_cb, problem.rig.wh)
        self.cvba_set_poses(problem.poses0 if poses is None else poses, problem.fixed_kf)
        self.cvba_set_landmarks(problem.lm0 if landmarks is None else landmarks)
        self.cvba_set_observations(problem.obs_kf, problem.obs_cam, problem.obs_lm, problem.obs_uv)
        return self


def cvba_evaluate_noalloc(n_obs: int, n_kf: int, n_cams: int, n_lm: int, intr: int, T_cb: int, T_bw: int, p_w: int,
                          kf: int, cam: int, lm: int, uv: int, huber_delta: float, z_min: float, out: int,
                          stream: int = 0) -> None:
    """Allocation-free cost evaluation from device pointers (see include/cvba.h); raises on a
    non-OK status.  `out` receives 5 doubles on the device, asynchronously on `stream`."""
    st = lib.cvba_evaluate_noalloc(int(n_obs), int(n_kf), int(n_cams), int(n_lm), C.c_void_p(intr),
                                   C.c_void_p(T_cb), C.c_void_p(T_bw), C.c_void_p(p_w), C.c_void_p(kf),
                                   C.c_void_p(cam), C.c_void_p(lm), C.c_void_p(uv), float(huber_delta),
                                   float(z_min), C.c_void_p(out), C.c_void_p(stream) if stream else None)
    if st != 0:
        raise CvbaError(st, "cvba_evaluate_noalloc failed")


def cvba_pnp_solve(dtype: int, n_frames: int, n_cams: int, n_lm: int, n_obs: int, intr: int, T_cb: int, p_w: int,
                   frame_off: int, cam: int, lm: int, uv: int, T_bw: int, iters: int, huber_delta: float = 1.0,
                   lambda0: float = 1e-4, z_min: float = 1e-3, trace: int = 0, stream: int = 0) -> None:
    """Motion-only bundle adjustment of a batch of frames from device pointers (see
    include/cvba.h); raises on a non-OK status.  dtype 0 = FP64, 1 = FP32 inputs."""
    o = make_opts(iters, huber_delta, lambda0, z_min)
    st = lib.cvba_pnp_solve(int(dtype), int(n_frames), int(n_cams), int(n_lm), int(n_obs), C.c_void_p(intr),
                            C.c_void_p(T_cb), C.c_void_p(p_w), C.c_void_p(frame_off), C.c_void_p(cam),
                            C.c_void_p(lm), C.c_void_p(uv), C.c_void_p(T_bw), C.byref(o),
                            C.c_void_p(trace) if trace else None, C.c_void_p(stream) if stream else None)
    if st != 0:
        raise CvbaError(st, "cvba_pnp_solve failed")


def cvba_relpose_solve(dtype: int, n_frames: int, n_cams: int, n_lm: int, n_obs: int, intr: int, T_cb: int,
                       p_w: int, frame_off: int, cam: int, lm: int, uv: int, T_mw: int, T_bm: int, iters: int,
                       huber_delta: float = 1.0, lambda0: float = 1e-4, z_min: float = 1e-3, trace: int = 0,
                       stream: int = 0) -> None:
    """Loop-closure relative poses of a batch of query frames from device pointers (see
    include/cvba.h); raises on a non-OK status."""
    o = make_opts(iters, huber_delta, lambda0, z_min)
    st = lib.cvba_relpose_solve(int(dtype), int(n_frames), int(n_cams), int(n_lm), int(n_obs), C.c_void_p(intr),
                                C.c_void_p(T_cb), C.c_void_p(p_w), C.c_void_p(frame_off), C.c_void_p(cam),
                                C.c_void_p(lm), C.c_void_p(uv), C.c_void_p(T_mw), C.c_void_p(T_bm), C.byref(o),
                                C.c_void_p(trace) if trace else None, C.c_void_p(stream) if stream else None)
    if st != 0:
        raise CvbaError(st, "cvba_relpose_solve failed")


def cvba_pgo_workspace_bytes(n_poses: int, n_edges: int) -> int:
    return int(lib.cvba_pgo_workspace_bytes(int(n_poses), int(n_edges)))


def cvba_pgo_solve(n_poses: int, n_edges: int, edges: int, deltas: int, poses: int, iters: int, fixed: int = 0,
                   lambda0: float = 1e-4, trace: int = 0, work: int = 0, work_bytes: int = 0, stream: int = 0) -> None:
    """Pose-graph optimisation from device pointers (see include/cvba.h); raises on a non-OK
    status."""
    o = make_opts(iters, 1.0, lambda0, 1e-3)
    st = lib.cvba_pgo_solve(int(n_poses), int(n_edges), C.c_void_p(edges), C.c_void_p(deltas), C.c_void_p(poses),
                            int(fixed), C.byref(o), C.c_void_p(trace) if trace else None, C.c_void_p(work),
                            int(work_bytes), C.c_void_p(stream) if stream else None)
    if st != 0:
        raise CvbaError(st, "cvba_pgo_solve failed")


def cvba_triangulate(dtype: int, n_lm: int, n_kf: int, n_cams: int, n_obs: int, intr: int, T_cb: int, T_bw: int,
                     lm_off: int, kf: int, cam: int, uv: int, p_w: int, iters: int, huber_delta: float = 1.0,
                     lambda0: float = 1e-4, z_min: float = 1e-3, p_lin: int = 0, status: int = 0, trace: int = 0,
                     stream: int = 0) -> None:
    """Multi-view triangulation of a batch of landmarks from device pointers (see
    include/cvba.h); raises on a non-OK status."""
    o = make_opts(iters, huber_delta, lambda0, z_min)
    opt = lambda x: C.c_void_p(x) if x else None
    st = lib.cvba_triangulate(int(dtype), int(n_lm), int(n_kf), int(n_cams), int(n_obs), C.c_void_p(intr),
                              C.c_void_p(T_cb), C.c_void_p(T_bw), C.c_void_p(lm_off), C.c_void_p(kf), C.c_void_p(cam),
                              C.c_void_p(uv), C.byref(o), opt(p_lin), C.c_void_p(p_w), opt(status), opt(trace),
                              opt(stream))
    if st != 0:
        raise CvbaError(st, "cvba_triangulate failed")


class Batch:
    """Independent windows solved together (cvba_batch_*): one launch per LM phase for all
    windows, one cluster per window for the Cholesky, the whole solve one CUDA graph."""

    def __init__(self, contexts):
        self.contexts = list(contexts)
        arr = (C.c_void_p * len(self.contexts))(*[c._h.value for c in self.contexts])
        h = C.c_void_p()
        st = lib.cvba_batch_create(C.byref(h), len(self.contexts), arr)
        if st != 0:
            raise CvbaError(st, "cvba_batch_create failed (same device and precision required)")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib.cvba_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _check(self, st):
        if st != 0:
            raise CvbaError(st, lib.cvba_batch_last_error(self._h).decode())

    def cvba_batch_solve(self, iters, huber_delta=1.0, lambda0=1e-4, z_min=1e-3, reset_lambda=True, refine=-1):
        o = make_opts(iters, huber_delta, lambda0, z_min, reset_lambda, refine)
        tr = np.zeros((len(self.contexts), max(int(iters), 1)), ITER_DTYPE)
        self._check(lib.cvba_batch_solve(self._h, C.byref(o), C.c_void_p(tr.ctypes.data)))
        return tr[:, :int(iters)]

    def cvba_batch_solve_async(self, iters, huber_delta=1.0, lambda0=1e-4, z_min=1e-3, reset_lambda=True, refine=-1):
        o = make_opts(iters, huber_delta, lambda0, z_min, reset_lambda, refine)
        self._check(lib.cvba_batch_solve_async(self._h, C.byref(o)))

    def cvba_batch_launch_count(self, iters, huber_delta=1.0, lambda0=1e-4, z_min=1e-3, refine=-1):
        o = make_opts(iters, huber_delta, lambda0, z_min, True, refine)
        n = C.c_int()
        self._check(lib.cvba_batch_launch_count(self._h, C.byref(o), C.byref(n)))
        return n.value

    def cvba_batch_set_chol_cluster(self, cs: int):
        self._check(lib.cvba_batch_set_chol_cluster(self._h, int(cs)))

    def cvba_batch_autotune(self, iters=2, huber_delta=1.0, lambda0=1e-4, z_min=1e-3, refine=-1):
        o = make_opts(iters, huber_delta, lambda0, z_min, True, refine)
        v = [C.c_int() for _ in range(3)]
        self._check(lib.cvba_batch_autotune(self._h, C.byref(o), *[C.byref(x) for x in v]))
        return dict(lin_tile_pairs=v[0].value, schur_tile_landmarks=v[1].value, chol_cluster=v[2].value)
