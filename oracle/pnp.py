"""Oracle for motion-only bundle adjustment (multi-camera PnP), one frame at a time.

TEST INFRASTRUCTURE ONLY (like oracle/ba.py): only tests/, __graft_entry__.smoke() and
bench.py's CPU legs may use it.  It shares no code with the CUDA library.

What it computes (cuVSLAM, arXiv 2506.04359): the pose estimate of a tracked frame,
Sec. 2.2.1 (stereo, Eq. PnP over the two cameras) and Sec. 2.2.2 (multi-stereo, the same
sum over every camera of the rig):
    T^bw = argmin  sum_j sum_k rho(|pi(T^cb_k T^bw p^w_j) - o_{j,k}|^2)
over the one base pose T^bw, with the landmarks p^w_j taken from the map and held fixed.
The residual, its Jacobian with respect to the left twist of T^bw, the Huber weights, the
Marquardt diagonal, Nielsen's damping update and the accept rule are the bundle-adjustment
oracle's (oracle/ba.py), restricted to one pose: the normal equations are the dense 6 x 6
system H = sum w J^T J, g = sum w J^T r, solved by Cholesky.  Exactly `iters` iterations.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import ba


def frame_window(intr, T_cb, lms, cam, lm, uv, huber_delta=1.0, z_min=1e-3) -> ba.Window:
    """A one-keyframe window holding a frame's observations (the keyframe index is 0)."""
    cam = np.asarray(cam, np.int64)
    return ba.Window(intr=np.asarray(intr, float), T_cb=np.asarray(T_cb, float).reshape(-1, 3, 4),
                     obs_kf=np.zeros(cam.size, np.int64), obs_cam=cam, obs_lm=np.asarray(lm, np.int64),
                     obs_uv=np.asarray(uv, float).reshape(-1, 2), K=1, M=int(np.asarray(lms).shape[0]),
                     fixed_kf=-1, huber_delta=huber_delta, z_min=z_min)


def normal_equations(w: ba.Window, T: np.ndarray, lms: np.ndarray):
    """H (6 x 6), g (6) over the frame's observations at pose T, and the evaluation."""
    r, valid = ba.residuals(w, T[None], lms)
    s = np.einsum("ni,ni->n", r, r)
    _, wt = ba.huber(s, w.huber_delta)
    wt = np.where(valid, wt, 0.0)
    Jp, _ = ba.jacobians(w, T[None], lms)
    H = np.einsum("n,nai,naj->ij", wt, Jp, Jp)
    g = np.einsum("n,nai,na->i", wt, Jp, r)
    return H, g, ba.evaluate(w, T[None], lms)


def lm_solve(w: ba.Window, T0: np.ndarray, lms: np.ndarray, iters: int, lam0: float = 1e-4):
    """Exactly `iters` LM iterations on the frame's pose; returns (T, lam, nu, trace)."""
    T, lam, nu = np.array(T0, float), lam0, 2.0
    lin = None
    trace = []
    for _ in range(iters):
        if lin is None:
            lin = normal_equations(w, T, lms)
        H, g, ev = lin
        D = ba.marquardt_diag(H)
        try:
            c = scipy.linalg.cho_factor(H + np.diag(lam * D), lower=True, check_finite=False)
            delta = scipy.linalg.cho_solve(c, -g, check_finite=False)
            ok = bool(np.all(np.isfinite(delta)))
        except np.linalg.LinAlgError:
            ok = False
        if not ok:
            trace.append(ba.IterRecord(ev.F, float("nan"), lam, float("nan"), float("nan"), float("nan"), False,
                                       ev.n_valid, ev.n_inlier, ev.rms, True, None))
            lam, nu = ba.nielsen_update(lam, nu, float("nan"), False)
            continue
        L = 0.5 * float(delta @ (lam * D * delta - g))
        T1 = ba.pose_plus(T, delta)
        F1 = ba.evaluate(w, T1[None], lms).F
        gain = (ev.F - F1) / L if L != 0.0 else float("nan")
        acc = ba.accept_step(L, F1, gain)
        trace.append(ba.IterRecord(ev.F, F1, lam, gain, L, float(np.linalg.norm(delta)), acc,
                                   ev.n_valid, ev.n_inlier, ev.rms, False, delta))
        lam, nu = ba.nielsen_update(lam, nu, gain, acc)
        if acc:
            T, lin = T1, None
    return T, lam, nu, trace


def solve_frames(batch, iters: int | None = None, frames=None, lam0: float = 1e-4, z_min: float = 1e-3):
    """Oracle solve of the selected frames of a synth.FrameBatch: list of (T, trace)."""
    iters = batch.iters if iters is None else iters
    out = []
    for f in (range(batch.F) if frames is None else frames):
        cam, lm, uv = batch.frame(f)
        w = frame_window(batch.rig.intr, batch.rig.T_cb, batch.lm, cam, lm, uv, batch.huber_delta, z_min)
        T, lam, nu, tr = lm_solve(w, batch.poses0[f], batch.lm, iters, lam0)
        out.append((T, tr))
    return out
