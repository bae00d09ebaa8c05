"""Oracle for multi-view landmark triangulation, one landmark at a time.

TEST INFRASTRUCTURE ONLY (like oracle/ba.py): only tests/, __graft_entry__.smoke() and
bench.py's CPU legs may use it.  It shares no code with the CUDA library.

What it computes (cuVSLAM, arXiv 2506.04359, Sec. 2.2 "3D module": on a new keyframe the
multi-view observations of new landmarks are triangulated, and the results become the
landmarks the bundle adjustment refines).  The paper names the step without a method; the
reading used here, for each landmark j with observations (keyframe i, camera k, pixel o):
  1. linear triangulation (inhomogeneous DLT, Hartley & Zisserman, "Multiple View
     Geometry", 2nd ed., Sec. 12.2): with x = ((u - cx)/fx, (v - cy)/fy) the normalised
     pixel and [R | t] = T^cb_k T^bw_i (camera from world), every observation gives the two
     linear equations  x (R_3 p + t_3) = R_1 p + t_1,  y (R_3 p + t_3) = R_2 p + t_2;
     p0 is their least-squares solution (numpy lstsq, an SVD solve);
  2. `iters` Levenberg-Marquardt iterations on the landmark alone, poses held fixed: the
     bundle-adjustment step of oracle/ba.py restricted to one landmark (Huber IRLS weights,
     Marquardt diagonal, Nielsen's damping update, accept iff L > 0 and gain > 0): the 3 x 3
     normal equations H = sum w J_lm^T J_lm, g = sum w J_lm^T r, solved by Cholesky.
A landmark with fewer than 2 observations, or whose linear system has rank < 3, is reported
invalid (status 1 / 2) and left at NaN.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import ba

STATUS_OK, STATUS_FEW_OBS, STATUS_DEGENERATE = 0, 1, 2


def camera_from_world(T_cb, poses, kf, cam):
    """[R | t] = T^cb_k T^bw_i for each observation: (n, 3, 3), (n, 3)."""
    Rc, tc = T_cb[cam, :, :3], T_cb[cam, :, 3]
    Rb, tb = poses[kf, :, :3], poses[kf, :, 3]
    R = np.einsum("nij,njk->nik", Rc, Rb)
    t = np.einsum("nij,nj->ni", Rc, tb) + tc
    return R, t


def linear(intr, T_cb, poses, kf, cam, uv):
    """Inhomogeneous DLT point of one landmark's observations, or None if rank < 3."""
    if len(kf) < 2:
        return None
    R, t = camera_from_world(T_cb, poses, kf, cam)
    f = intr[cam]
    x = (uv[:, 0] - f[:, 2]) / f[:, 0]
    y = (uv[:, 1] - f[:, 3]) / f[:, 1]
    A = np.concatenate([x[:, None] * R[:, 2] - R[:, 0], y[:, None] * R[:, 2] - R[:, 1]], 0)
    b = np.concatenate([t[:, 0] - x * t[:, 2], t[:, 1] - y * t[:, 2]], 0)
    p, _, rank, _ = np.linalg.lstsq(A, b, rcond=None)
    return p if rank == 3 else None


def landmark_window(intr, T_cb, kf, cam, uv, K, huber_delta, z_min):
    """A window holding one landmark's observations (landmark index 0)."""
    kf = np.asarray(kf, np.int64)
    return ba.Window(intr=np.asarray(intr, float), T_cb=np.asarray(T_cb, float), obs_kf=kf,
                     obs_cam=np.asarray(cam, np.int64), obs_lm=np.zeros(kf.size, np.int64),
                     obs_uv=np.asarray(uv, float).reshape(-1, 2), K=K, M=1, fixed_kf=-1,
                     huber_delta=huber_delta, z_min=z_min)


def refine(w: ba.Window, poses, p0, iters: int, lam0: float = 1e-4):
    """Exactly `iters` LM iterations on the landmark; returns (p, trace)."""
    p, lam, nu = np.array(p0, float), lam0, 2.0
    lin = None
    trace = []
    for _ in range(iters):
        if lin is None:
            r, valid = ba.residuals(w, poses, p[None])
            s = np.einsum("ni,ni->n", r, r)
            _, wt = ba.huber(s, w.huber_delta)
            wt = np.where(valid, wt, 0.0)
            _, Jl = ba.jacobians(w, poses, p[None])
            H = np.einsum("n,nai,naj->ij", wt, Jl, Jl)
            g = np.einsum("n,nai,na->i", wt, Jl, r)
            lin = (H, g, ba.evaluate(w, poses, p[None]))
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
        p1 = p + delta
        F1 = ba.evaluate(w, poses, p1[None]).F
        gain = (ev.F - F1) / L if L != 0.0 else float("nan")
        acc = ba.accept_step(L, F1, gain)
        trace.append(ba.IterRecord(ev.F, F1, lam, gain, L, float(np.linalg.norm(delta)), acc,
                                   ev.n_valid, ev.n_inlier, ev.rms, False, delta))
        lam, nu = ba.nielsen_update(lam, nu, gain, acc)
        if acc:
            p, lin = p1, None
    return p, trace


def triangulate(intr, T_cb, poses, lm_off, kf, cam, uv, iters: int, huber_delta: float = 1.0,
                z_min: float = 1e-3, lam0: float = 1e-4, landmarks=None):
    """Triangulate the selected landmarks (observations of landmark j: [lm_off[j], lm_off[j+1])).
    Returns (p0 linear, p refined, status, traces) for each selected landmark."""
    intr, T_cb, poses = np.asarray(intr, float), np.asarray(T_cb, float).reshape(-1, 3, 4), np.asarray(poses, float)
    out = []
    for j in (range(len(lm_off) - 1) if landmarks is None else landmarks):
        a, b = int(lm_off[j]), int(lm_off[j + 1])
        k_, c_, o_ = np.asarray(kf[a:b], np.int64), np.asarray(cam[a:b], np.int64), np.asarray(uv[a:b], float)
        if b - a < 2:
            out.append((np.full(3, np.nan), np.full(3, np.nan), STATUS_FEW_OBS, []))
            continue
        p0 = linear(intr, T_cb, poses, k_, c_, o_)
        if p0 is None:
            out.append((np.full(3, np.nan), np.full(3, np.nan), STATUS_DEGENERATE, []))
            continue
        w = landmark_window(intr, T_cb, k_, c_, o_, poses.shape[0], huber_delta, z_min)
        p, tr = refine(w, poses, p0, iters, lam0)
        out.append((p0, p, STATUS_OK, tr))
    return out
