"""Plain FP64 CPU oracle for one sliding-window bundle-adjustment LM solve.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import or call this module:
only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference leg use it.
It shares no code with the CUDA library (paper_2506_04359_gb300/csrc) and imports nothing
from it.

What it computes (cuVSLAM, arXiv 2506.04359, Sec. 2.2 "3D module"):
  * reprojection residual  r_n = pi(T^cb_k T^bw_i p^w_j) - o_{j,k}         (Eq. r^repr)
  * objective              F = 1/2 sum_n rho(||r_n||^2)                    (Eq. argmin,
    with Sigma = I and a Huber kernel rho of threshold delta on the per-observation norm)
The paper states the problem and says the solve eliminates landmarks with the Schur
complement.  That elimination is an exact rewrite of one linear solve, so this oracle does
NOT use it: it assembles the full dense normal equations over all free pose and landmark
coordinates and factors them with a dense Cholesky (LAPACK via scipy), i.e. the plain
definition of the damped Gauss-Newton step.  The LM iteration itself is taken step by
step in the order given below.

Readings where the paper is silent (all fixed here and in the CUDA library alike):
  pinhole projection without distortion; Sigma = I (pixels); Huber weight w = 1 for
  ||r|| <= delta and delta/||r|| otherwise (IRLS, weights held at the linearisation
  point); left SE(3) update T <- Exp(xi) T with xi = (rho, phi), translation first;
  Euclidean landmark update p <- p + dp; keyframe `fixed_kf` removed (gauge);
  observations with camera depth Z <= z_min are invalid (no cost, no Jacobian);
  Marquardt scaling D = diag(H) floored at 1e-12 * max(diag H); Nielsen's lambda update;
  a step is accepted iff the predicted reduction L > 0 and the gain ratio > 0; exactly
  `iters` iterations, each with one linear solve, accepted or not.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg

TAYLOR_THETA = 1e-4     # below this rotation angle Exp uses its Taylor series
DIAG_FLOOR = 1e-12      # Marquardt diagonal floor, relative to max(diag H)


# --------------------------------------------------------------------------- SE(3)

def hat(v: np.ndarray) -> np.ndarray:
    """Skew-symmetric matrix [v]x with [v]x w = v x w."""
    x, y, z = v
    return np.array([[0.0, -z, y], [z, 0.0, -x], [-y, x, 0.0]])


def so3_exp(phi: np.ndarray) -> np.ndarray:
    """Rodrigues: R = I + A [phi]x + B [phi]x^2, A = sin t / t, B = (1 - cos t) / t^2."""
    t = float(np.linalg.norm(phi))
    if t < TAYLOR_THETA:
        A = 1.0 - t * t / 6.0
        B = 0.5 - t * t / 24.0
    else:
        A = math.sin(t) / t
        B = (1.0 - math.cos(t)) / (t * t)
    P = hat(phi)
    return np.eye(3) + A * P + B * (P @ P)


def se3_exp(xi: np.ndarray):
    """Exp of the twist xi = (rho, phi): (R, t) with t = V rho,
    V = I + B [phi]x + C [phi]x^2, C = (t - sin t) / t^3."""
    rho, phi = xi[:3], xi[3:]
    t = float(np.linalg.norm(phi))
    if t < TAYLOR_THETA:
        B = 0.5 - t * t / 24.0
        C = 1.0 / 6.0 - t * t / 120.0
    else:
        B = (1.0 - math.cos(t)) / (t * t)
        C = (t - math.sin(t)) / (t ** 3)
    P = hat(phi)
    V = np.eye(3) + B * P + C * (P @ P)
    return so3_exp(phi), V @ rho


def pose_plus(T: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """Left update Exp(xi) * T for a (3, 4) pose [R | t]."""
    Re, te = se3_exp(xi)
    out = np.empty((3, 4))
    out[:, :3] = Re @ T[:, :3]
    out[:, 3] = Re @ T[:, 3] + te
    return out


# -------------------------------------------------------------------------- model

@dataclass
class Window:
    """One BA window: rig, observations and settings (state lives outside)."""
    intr: np.ndarray       # (C, 4)
    T_cb: np.ndarray       # (C, 3, 4)
    obs_kf: np.ndarray     # (N,)
    obs_cam: np.ndarray    # (N,)
    obs_lm: np.ndarray     # (N,)
    obs_uv: np.ndarray     # (N, 2)
    K: int
    M: int
    fixed_kf: int = 0
    huber_delta: float = 1.0
    z_min: float = 1e-3

    @classmethod
    def from_problem(cls, p, huber_delta=None, z_min=1e-3) -> "Window":
        return cls(intr=np.asarray(p.rig.intr, float), T_cb=np.asarray(p.rig.T_cb, float),
                   obs_kf=np.asarray(p.obs_kf, np.int64), obs_cam=np.asarray(p.obs_cam, np.int64),
                   obs_lm=np.asarray(p.obs_lm, np.int64), obs_uv=np.asarray(p.obs_uv, float),
                   K=p.K, M=p.M, fixed_kf=p.fixed_kf,
                   huber_delta=p.huber_delta if huber_delta is None else huber_delta, z_min=z_min)

    @property
    def free_kfs(self) -> np.ndarray:
        return np.array([i for i in range(self.K) if i != self.fixed_kf], np.int64)

    @property
    def n_c(self) -> int:
        return 6 * (self.K - 1)

    @property
    def n_f(self) -> int:
        return self.n_c + 3 * self.M

    def pose_col(self) -> np.ndarray:
        """First column of each keyframe's 6 pose columns; -1 for the fixed keyframe."""
        col = -np.ones(self.K, np.int64)
        col[self.free_kfs] = 6 * np.arange(self.K - 1)
        return col


def transform(win: Window, poses: np.ndarray, lms: np.ndarray):
    """X_b = R_i p_j + t_i and X_c = R^cb_k X_b + t^cb_k for every observation."""
    R = poses[win.obs_kf, :, :3]
    t = poses[win.obs_kf, :, 3]
    Xb = np.einsum("nij,nj->ni", R, lms[win.obs_lm]) + t
    Rc = win.T_cb[win.obs_cam, :, :3]
    tc = win.T_cb[win.obs_cam, :, 3]
    Xc = np.einsum("nij,nj->ni", Rc, Xb) + tc
    return Xb, Xc


def residuals(win: Window, poses: np.ndarray, lms: np.ndarray):
    """r (N, 2) = pi(X_c) - o and the validity mask Z_c > z_min (invalid rows set to 0)."""
    _, Xc = transform(win, poses, lms)
    Z = Xc[:, 2]
    valid = Z > win.z_min
    Zs = np.where(valid, Z, 1.0)
    f = win.intr[win.obs_cam]
    u = f[:, 0] * Xc[:, 0] / Zs + f[:, 2]
    v = f[:, 1] * Xc[:, 1] / Zs + f[:, 3]
    r = np.stack([u, v], 1) - win.obs_uv
    r[~valid] = 0.0
    return r, valid


def huber(s: np.ndarray, delta: float):
    """rho(s) on the squared norm s, and the IRLS weight w = d rho / d s."""
    e = np.sqrt(s)
    inl = e <= delta
    rho = np.where(inl, s, 2.0 * delta * e - delta * delta)
    w = np.where(inl, 1.0, delta / np.where(inl, 1.0, e))
    return rho, w


def jacobians(win: Window, poses: np.ndarray, lms: np.ndarray):
    """Per-observation J_pose (N, 2, 6) w.r.t. the left twist of T^bw_i and J_lm (N, 2, 3).

    dX_b/dxi = [I | -[X_b]x],  dX_b/dp = R_i,  dX_c/dX_b = R^cb_k,
    dpi/dX_c = [[fx/Z, 0, -fx X/Z^2], [0, fy/Z, -fy Y/Z^2]]."""
    Xb, Xc = transform(win, poses, lms)
    N = Xc.shape[0]
    X, Y, Z = Xc[:, 0], Xc[:, 1], np.where(Xc[:, 2] > win.z_min, Xc[:, 2], 1.0)
    f = win.intr[win.obs_cam]
    Jpi = np.zeros((N, 2, 3))
    Jpi[:, 0, 0] = f[:, 0] / Z
    Jpi[:, 0, 2] = -f[:, 0] * X / (Z * Z)
    Jpi[:, 1, 1] = f[:, 1] / Z
    Jpi[:, 1, 2] = -f[:, 1] * Y / (Z * Z)
    Rc = win.T_cb[win.obs_cam, :, :3]
    dXb = np.zeros((N, 3, 6))
    dXb[:, :, :3] = np.eye(3)
    # -[X_b]x, row by row
    dXb[:, 0, 4], dXb[:, 0, 5] = Xb[:, 2], -Xb[:, 1]
    dXb[:, 1, 3], dXb[:, 1, 5] = -Xb[:, 2], Xb[:, 0]
    dXb[:, 2, 3], dXb[:, 2, 4] = Xb[:, 1], -Xb[:, 0]
    JpR = np.einsum("nij,njk->nik", Jpi, Rc)
    Jpose = np.einsum("nij,njk->nik", JpR, dXb)
    Jlm = np.einsum("nij,njk->nik", JpR, poses[win.obs_kf, :, :3])
    return Jpose, Jlm


@dataclass
class Eval:
    F: float
    n_valid: int
    n_inlier: int
    rms: float


def evaluate(win: Window, poses, lms) -> Eval:
    """F = 1/2 sum rho(||r||^2) over valid observations; counts; unweighted RMS in px."""
    r, valid = residuals(win, poses, lms)
    s = np.einsum("ni,ni->n", r, r)
    rho, _ = huber(s, win.huber_delta)
    n_valid = int(valid.sum())
    n_inl = int((valid & (np.sqrt(s) <= win.huber_delta)).sum())
    F = 0.5 * float(rho[valid].sum())
    rms = math.sqrt(float(s[valid].sum()) / n_valid) if n_valid else 0.0
    return Eval(F, n_valid, n_inl, rms)


def normal_equations(win: Window, poses, lms):
    """Dense H = sum_n w_n J_n^T J_n and g = sum_n w_n J_n^T r_n over all free columns
    (free keyframe twists in index order, then landmarks), plus the evaluation at x."""
    r, valid = residuals(win, poses, lms)
    s = np.einsum("ni,ni->n", r, r)
    _, w = huber(s, win.huber_delta)
    w = np.where(valid, w, 0.0)
    Jp, Jl = jacobians(win, poses, lms)
    N = r.shape[0]
    J = np.concatenate([Jp, Jl], axis=2)                         # (N, 2, 9)
    pc = win.pose_col()[win.obs_kf]
    dummy = win.n_f                                              # fixed-keyframe columns land here
    cols = np.empty((N, 9), np.int64)
    cols[:, :6] = np.where(pc[:, None] >= 0, pc[:, None] + np.arange(6), dummy)
    cols[:, 6:] = win.n_c + 3 * win.obs_lm[:, None] + np.arange(3)
    blocks = w[:, None, None] * np.einsum("nai,naj->nij", J, J)  # (N, 9, 9)
    gblk = w[:, None] * np.einsum("nai,na->ni", J, r)            # (N, 9)
    H = np.zeros((win.n_f + 1, win.n_f + 1))
    g = np.zeros(win.n_f + 1)
    np.add.at(H, (np.repeat(cols, 9, axis=1), np.tile(cols, (1, 9))), blocks.reshape(N, 81))
    np.add.at(g, cols, gblk)
    return H[:-1, :-1], g[:-1], evaluate(win, poses, lms)


def marquardt_diag(H: np.ndarray) -> np.ndarray:
    d = np.diag(H).copy()
    floor = DIAG_FLOOR * (d.max() if d.size else 0.0)
    return np.maximum(d, floor)


def damped_solve(H: np.ndarray, g: np.ndarray, lam: float):
    """delta solving (H + lam D) delta = -g by dense Cholesky; None if not positive definite."""
    D = marquardt_diag(H)
    A = H + np.diag(lam * D)
    try:
        c = scipy.linalg.cho_factor(A, lower=True, overwrite_a=True, check_finite=False)
    except np.linalg.LinAlgError:
        return None, D
    delta = scipy.linalg.cho_solve(c, -g, check_finite=False)
    if not np.all(np.isfinite(delta)):
        return None, D
    return delta, D


def apply_step(win: Window, poses, lms, delta):
    """x (+) delta: left SE(3) update on free keyframes, Euclidean update on landmarks."""
    out_p = poses.copy()
    for n, i in enumerate(win.free_kfs):
        out_p[i] = pose_plus(poses[i], delta[6 * n: 6 * n + 6])
    out_l = lms + delta[win.n_c:].reshape(win.M, 3)
    return out_p, out_l


# ---------------------------------------------------------------------------- LM

@dataclass
class IterRecord:
    cost0: float          # F at the linearisation point
    cost1: float          # F at the candidate (nan if the system was not PD)
    lam: float            # lambda used for this solve
    gain: float           # (F - F') / L
    pred: float           # L = 1/2 delta^T (lam D delta - g)
    step_norm: float
    accepted: bool
    n_valid: int
    n_inlier: int
    rms: float
    nonpd: bool
    delta: np.ndarray | None


def accept_step(L: float, F1: float, gain: float) -> bool:
    """A candidate is accepted iff the predicted reduction L is positive, its cost is finite
    and the gain ratio (F - F') / L is positive."""
    return bool(L > 0.0 and np.isfinite(F1) and gain > 0.0)


def nielsen_update(lam: float, nu: float, gain: float, accepted: bool):
    """Nielsen's damping update (H. B. Nielsen, "Damping parameter in Marquardt's method",
    IMM-REP-1999-05): after an accepted step lambda <- lambda * max(1/3, 1 - (2 gain - 1)^3)
    and nu <- 2; after a rejected (or not positive definite) step lambda <- lambda * nu and
    nu <- 2 nu."""
    if accepted:
        return lam * max(1.0 / 3.0, 1.0 - (2.0 * gain - 1.0) ** 3), 2.0
    return lam * nu, 2.0 * nu


def lm_iteration(win: Window, poses, lms, lam, nu, lin=None):
    """One LM iteration from state x with damping (lam, nu).

    Returns (poses', lms', lam', nu', record, lin') where lin' is the linearisation at the
    returned state (reused by the caller when the step was rejected)."""
    if lin is None:
        lin = normal_equations(win, poses, lms)
    H, g, ev = lin
    delta, D = damped_solve(H, g, lam)
    if delta is None:
        rec = IterRecord(ev.F, float("nan"), lam, float("nan"), float("nan"), float("nan"), False,
                         ev.n_valid, ev.n_inlier, ev.rms, True, None)
        lam_new, nu_new = nielsen_update(lam, nu, float("nan"), False)
        return poses, lms, lam_new, nu_new, rec, lin
    L = 0.5 * float(delta @ (lam * D * delta - g))
    p1, l1 = apply_step(win, poses, lms, delta)
    F1 = evaluate(win, p1, l1).F
    gain = (ev.F - F1) / L if L != 0.0 else float("nan")
    acc = accept_step(L, F1, gain)
    rec = IterRecord(ev.F, F1, lam, gain, L, float(np.linalg.norm(delta)), acc,
                     ev.n_valid, ev.n_inlier, ev.rms, False, delta)
    lam_new, nu_new = nielsen_update(lam, nu, gain, acc)
    if acc:
        return p1, l1, lam_new, nu_new, rec, None
    return poses, lms, lam_new, nu_new, rec, lin


def lm_solve(win: Window, poses0, lms0, iters: int, lam0: float = 1e-4, keep_delta: bool = True):
    """Exactly `iters` LM iterations; returns final (poses, lms, lam, nu) and the trace."""
    poses, lms, lam, nu = poses0.copy(), lms0.copy(), lam0, 2.0
    lin = None
    trace = []
    for _ in range(iters):
        poses, lms, lam, nu, rec, lin = lm_iteration(win, poses, lms, lam, nu, lin)
        if not keep_delta:
            rec.delta = None
        trace.append(rec)
    return poses, lms, lam, nu, trace


# ------------------------------------------------------------------ checks / layout

def normal_residual(win: Window, poses, lms, lam, delta):
    """|| (H + lam D) delta + g || / ||g|| computed matrix-free per observation, for
    windows too large for the dense system.  D uses the same floored diagonal."""
    r, valid = residuals(win, poses, lms)
    s = np.einsum("ni,ni->n", r, r)
    _, w = huber(s, win.huber_delta)
    w = np.where(valid, w, 0.0)
    Jp, Jl = jacobians(win, poses, lms)
    pc = win.pose_col()[win.obs_kf]
    dpose = np.zeros((r.shape[0], 6))
    free = pc >= 0
    dpose[free] = delta[pc[free][:, None] + np.arange(6)]
    dl = delta[win.n_c:].reshape(win.M, 3)[win.obs_lm]
    Jd = np.einsum("nij,nj->ni", Jp, dpose) + np.einsum("nij,nj->ni", Jl, dl)
    y = w[:, None] * (Jd + r)                                # w (J delta + r)
    out = np.zeros(win.n_f + 1)
    diag = np.zeros(win.n_f + 1)
    cols_p = np.where(free[:, None], pc[:, None] + np.arange(6), win.n_f)
    cols_l = win.n_c + 3 * win.obs_lm[:, None] + np.arange(3)
    np.add.at(out, cols_p, np.einsum("nai,na->ni", Jp, y))
    np.add.at(out, cols_l, np.einsum("nai,na->ni", Jl, y))
    np.add.at(diag, cols_p, w[:, None] * np.einsum("nai,nai->ni", Jp, Jp))
    np.add.at(diag, cols_l, w[:, None] * np.einsum("nai,nai->ni", Jl, Jl))
    d = diag[:-1]
    D = np.maximum(d, DIAG_FLOOR * d.max())
    res = out[:-1] + lam * D * delta                            # H delta + g + lam D delta
    gvec = np.zeros(win.n_f + 1)
    np.add.at(gvec, cols_p, w[:, None] * np.einsum("nai,na->ni", Jp, r))
    np.add.at(gvec, cols_l, w[:, None] * np.einsum("nai,na->ni", Jl, r))
    return float(np.linalg.norm(res) / np.linalg.norm(gvec[:-1]))


def layout(obs_kf, obs_cam, obs_lm, M):
    """Stable sort of observations by (landmark, keyframe, camera) and landmark offsets."""
    perm = np.lexsort((obs_cam, obs_kf, obs_lm)).astype(np.int32)
    counts = np.bincount(np.asarray(obs_lm, np.int64), minlength=M)
    lm_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    return perm, lm_off


def device_layout(obs_kf, obs_cam, obs_lm, M):
    """Integer layout the library builds, by its definition: landmarks ordered by (first
    observing keyframe, last observing keyframe, caller index); observation slots ordered
    by (landmark rank, keyframe, camera, caller index); landmark segment offsets."""
    obs_kf = np.asarray(obs_kf, np.int64)
    obs_lm = np.asarray(obs_lm, np.int64)
    first = np.full(M, np.iinfo(np.int64).max)
    last = np.full(M, -1)
    np.minimum.at(first, obs_lm, obs_kf)
    np.maximum.at(last, obs_lm, obs_kf)
    lm_order = np.lexsort((np.arange(M), last, first)).astype(np.int32)
    rank = np.empty(M, np.int64)
    rank[lm_order] = np.arange(M)
    n = np.arange(obs_kf.size)
    obs_order = np.lexsort((n, np.asarray(obs_cam, np.int64), obs_kf, rank[obs_lm])).astype(np.int32)
    counts = np.bincount(rank[obs_lm], minlength=M)
    lm_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    return lm_order, obs_order, lm_off


# --------------------------------------------------------------- differentiable cost

def se3_left_jacobian(xi: np.ndarray) -> np.ndarray:
    """Left Jacobian of SE(3) at xi = (rho, phi): Exp(xi + d) ~ Exp(J_l d) Exp(xi).
    J_l = [[J, Q], [0, J]] with J the SO(3) left Jacobian (= V of se3_exp) and Q(rho, phi)
    the closed form of Barfoot, State Estimation for Robotics (2017), Eq. (7.86)."""
    rho, phi = xi[:3], xi[3:]
    t = float(np.linalg.norm(phi))
    if t < TAYLOR_THETA:
        B, C = 0.5 - t * t / 24.0, 1.0 / 6.0 - t * t / 120.0
        D, E = 1.0 / 24.0 - t * t / 720.0, 1.0 / 120.0 - t * t / 2520.0
    else:
        B = (1.0 - math.cos(t)) / (t * t)
        C = (t - math.sin(t)) / t ** 3
        D = (t * t + 2.0 * math.cos(t) - 2.0) / (2.0 * t ** 4)
        E = (2.0 * t - 3.0 * math.sin(t) + t * math.cos(t)) / (2.0 * t ** 5)
    P, R = hat(phi), hat(rho)
    J = np.eye(3) + B * P + C * (P @ P)
    Q = (0.5 * R + C * (P @ R + R @ P + P @ R @ P) + D * (P @ P @ R + R @ P @ P - 3.0 * P @ R @ P)
         + E * (P @ R @ P @ P + P @ P @ R @ P))
    out = np.zeros((6, 6))
    out[:3, :3] = J
    out[:3, 3:] = Q
    out[3:, 3:] = J
    return out


def cost_grad(win: Window, poses, lms, intr=None, xi=None):
    """F = 1/2 sum rho(|r|^2) with keyframe i at Exp(xi_i) T_i, and its gradient w.r.t.
    xi (K, 6), the pose matrices T (K, 3, 4), the landmarks (M, 3) and the intrinsics (C, 4).

    dF/dxi_i = J_l(xi_i)^T sum_n J_pose,n^T w_n r_n   (J_pose: left perturbation at T')
    dF/dT_i  = sum_n R_e^T g_X (x) [p_j; 1],  g_X = (dr/dX')^T w r
    dF/dp_j  = sum_n J_lm,n^T w_n r_n
    dF/dintr = sum_n w (r_u X/Z, r_v Y/Z, r_u, r_v)."""
    K, M = win.K, win.M
    intr = win.intr if intr is None else np.asarray(intr, float)
    xi = np.zeros((K, 6)) if xi is None else np.asarray(xi, float)
    Tp = np.stack([pose_plus(poses[i], xi[i]) for i in range(K)])
    w2 = Window(intr=intr, T_cb=win.T_cb, obs_kf=win.obs_kf, obs_cam=win.obs_cam, obs_lm=win.obs_lm,
                obs_uv=win.obs_uv, K=K, M=M, fixed_kf=-1, huber_delta=win.huber_delta, z_min=win.z_min)
    r, valid = residuals(w2, Tp, lms)
    s = np.einsum("ni,ni->n", r, r)
    rho, w = huber(s, win.huber_delta)
    w = np.where(valid, w, 0.0)
    F = 0.5 * float(rho[valid].sum())
    Jp, Jl = jacobians(w2, Tp, lms)
    wr = w[:, None] * r
    g_left = np.zeros((K, 6))
    np.add.at(g_left, win.obs_kf, np.einsum("nai,na->ni", Jp, wr))
    g_xi = np.stack([se3_left_jacobian(xi[i]).T @ g_left[i] for i in range(K)])
    g_lm = np.zeros((M, 3))
    np.add.at(g_lm, win.obs_lm, np.einsum("nai,na->ni", Jl, wr))
    # dr/dX' = J_pi R_cb; g_X = (dr/dX')^T w r; dX'/dR_ab = R_e[:, a] p_b, dX'/dt = R_e
    Xb, Xc = transform(w2, Tp, lms)
    Zs = np.where(valid, Xc[:, 2], 1.0)
    f = intr[win.obs_cam]
    Jpi = np.zeros((r.shape[0], 2, 3))
    Jpi[:, 0, 0] = f[:, 0] / Zs
    Jpi[:, 0, 2] = -f[:, 0] * Xc[:, 0] / Zs ** 2
    Jpi[:, 1, 1] = f[:, 1] / Zs
    Jpi[:, 1, 2] = -f[:, 1] * Xc[:, 1] / Zs ** 2
    dXc = np.einsum("nai,na->ni", Jpi, wr)
    gX = np.einsum("nji,nj->ni", win.T_cb[win.obs_cam, :, :3], dXc)
    Re = np.stack([Tp[i, :, :3] @ poses[i, :, :3].T for i in range(K)])
    h = np.einsum("nji,nj->ni", Re[win.obs_kf], gX)
    p1 = np.concatenate([lms[win.obs_lm], np.ones((r.shape[0], 1))], axis=1)
    g_T = np.zeros((K, 3, 4))
    np.add.at(g_T, win.obs_kf, h[:, :, None] * p1[:, None, :])
    g_intr = np.zeros_like(intr)
    terms = np.stack([wr[:, 0] * Xc[:, 0] / Zs, wr[:, 1] * Xc[:, 1] / Zs, wr[:, 0], wr[:, 1]], 1)
    np.add.at(g_intr, win.obs_cam, terms)
    return F, dict(xi=g_xi, T=g_T, lm=g_lm, intr=g_intr)
