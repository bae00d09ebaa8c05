"""Oracle for pose-graph optimisation (PGO), the dense plain form.

TEST INFRASTRUCTURE ONLY (like oracle/ba.py): only tests/, __graft_entry__.smoke() and
bench.py's CPU legs may use it.  It shares no code with the CUDA library.

What it computes (cuVSLAM, arXiv 2506.04359, Sec. 2.3, Eq. PGO): given pose deltas D_ij on
the edges E of a pose graph (from frontend odometry or loop closures),
    T_{1:N} = argmin  sum_{(i,j) in E} |Log(D_ij^-1 T_i^-1 T_j)|^2 .
Readings (the paper fixes none of them): T_i is the keyframe's world-from-base pose, so that
T_i^-1 T_j is the pose of j in i's frame, which the delta D_ij measures; Log is the SE(3)
logarithm with the twist (rho, phi), translation first, the inverse of the Exp of the window
solve; the norm is plain (no weights, no robust kernel); one pose is held fixed (the gauge);
poses are updated on the left, T_i <- Exp(xi_i) T_i.  With E = D^-1 T_i^-1 T_j and
r = Log(E), left perturbations give E Exp(Ad(T_j^-1) xi_j) and E Exp(-Ad(T_j^-1) xi_i), so
    dr/dxi_j = J_r(r)^-1 Ad(T_j^-1),   dr/dxi_i = -dr/dxi_j,
with J_r(xi) = J_l(-xi) the right Jacobian of SE(3) (J_l: oracle/ba.py's closed form,
Barfoot 2017, Eq. 7.86) and Ad(T) = [[R, [t]x R], [0, R]].  The LM iteration is the window
solve's: H = sum J^T J, g = sum J^T r (dense over the free poses), D = diag(H) floored at
1e-12 max, (H + lambda D) delta = -g by Cholesky, F = 1/2 sum |r|^2, Nielsen's damping
update, accept iff L > 0 and gain > 0, exactly `iters` iterations.  Iteration records count
every edge as valid and as an inlier (there is no robust kernel) and report the RMS edge
residual sqrt(2 F / |E|).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

from . import ba

TAYLOR_THETA = 1e-4


def so3_log(R: np.ndarray) -> np.ndarray:
    """phi with Exp(phi) = R: theta = acos((tr R - 1) / 2), phi = theta / (2 sin theta) vee(R - R^T);
    series below theta = 1e-4; near theta = pi the axis from the largest diagonal entry."""
    c = float(np.clip((np.trace(R) - 1.0) / 2.0, -1.0, 1.0))
    w = np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    theta = math.acos(c)
    if theta < TAYLOR_THETA:
        return 0.5 * (1.0 + theta * theta / 6.0) * w
    if math.pi - theta < 1e-6:
        B = (R + np.eye(3)) / 2.0
        k = int(np.argmax(np.diag(B)))
        axis = B[:, k] / math.sqrt(B[k, k])
        if np.dot(axis, w) < 0:
            axis = -axis
        return theta * axis / np.linalg.norm(axis)
    return theta / (2.0 * math.sin(theta)) * w


def se3_log(T: np.ndarray) -> np.ndarray:
    """xi = (rho, phi) with Exp(xi) = T: phi = Log(R), rho = V(phi)^-1 t."""
    phi = so3_log(T[:, :3])
    Jl = ba.se3_left_jacobian(np.concatenate([np.zeros(3), phi]))
    V = Jl[:3, :3]
    return np.concatenate([np.linalg.solve(V, T[:, 3]), phi])


def inverse(T):
    out = np.empty((3, 4))
    out[:, :3] = T[:, :3].T
    out[:, 3] = -T[:, :3].T @ T[:, 3]
    return out


def compose(A, B):
    out = np.empty((3, 4))
    out[:, :3] = A[:, :3] @ B[:, :3]
    out[:, 3] = A[:, :3] @ B[:, 3] + A[:, 3]
    return out


def adjoint(T: np.ndarray) -> np.ndarray:
    R, t = T[:, :3], T[:, 3]
    out = np.zeros((6, 6))
    out[:3, :3] = R
    out[:3, 3:] = ba.hat(t) @ R
    out[3:, 3:] = R
    return out


def edge_residual(Ti, Tj, D):
    """r = Log(D^-1 T_i^-1 T_j)."""
    return se3_log(compose(inverse(D), compose(inverse(Ti), Tj)))


def edge_jacobians(Ti, Tj, D):
    """(r, dr/dxi_i, dr/dxi_j) for left perturbations of T_i and T_j."""
    r = edge_residual(Ti, Tj, D)
    Jr_inv = np.linalg.inv(ba.se3_left_jacobian(-r))
    Jj = Jr_inv @ adjoint(inverse(Tj))
    return r, -Jj, Jj


def cost(poses, edges, deltas) -> float:
    return 0.5 * sum(float(r @ r) for r in (edge_residual(poses[i], poses[j], D)
                                            for (i, j), D in zip(edges, deltas)))


def normal_equations(poses, edges, deltas, fixed: int = 0):
    """Dense H, g over the free poses (index order, the fixed one removed) and the cost."""
    K = poses.shape[0]
    col = -np.ones(K, np.int64)
    col[[k for k in range(K) if k != fixed]] = 6 * np.arange(K - 1)
    n = 6 * (K - 1)
    H, g, F = np.zeros((n, n)), np.zeros(n), 0.0
    for (i, j), D in zip(edges, deltas):
        r, Ji, Jj = edge_jacobians(poses[i], poses[j], D)
        F += 0.5 * float(r @ r)
        for a, Ja in ((i, Ji), (j, Jj)):
            if col[a] < 0:
                continue
            g[col[a]:col[a] + 6] += Ja.T @ r
            for b, Jb in ((i, Ji), (j, Jj)):
                if col[b] >= 0:
                    H[col[a]:col[a] + 6, col[b]:col[b] + 6] += Ja.T @ Jb
    return H, g, F, col


def apply_step(poses, delta, col):
    out = poses.copy()
    for k in range(poses.shape[0]):
        if col[k] >= 0:
            out[k] = ba.pose_plus(poses[k], delta[col[k]:col[k] + 6])
    return out


def lm_solve(poses0, edges, deltas, iters: int, lam0: float = 1e-4, fixed: int = 0):
    """Exactly `iters` LM iterations; returns (poses, lam, nu, trace)."""
    poses, lam, nu = np.array(poses0, float), lam0, 2.0
    lin = None
    trace = []
    for _ in range(iters):
        if lin is None:
            lin = normal_equations(poses, edges, deltas, fixed)
        H, g, F, col = lin
        D = ba.marquardt_diag(H)
        try:
            c = scipy.linalg.cho_factor(H + np.diag(lam * D), lower=True, check_finite=False)
            delta = scipy.linalg.cho_solve(c, -g, check_finite=False)
            ok = bool(np.all(np.isfinite(delta)))
        except np.linalg.LinAlgError:
            ok = False
        if not ok:
            trace.append(ba.IterRecord(F, float("nan"), lam, float("nan"), float("nan"), float("nan"), False,
                                       len(edges), len(edges), math.sqrt(2.0 * F / len(edges)), True, None))
            lam, nu = ba.nielsen_update(lam, nu, float("nan"), False)
            continue
        L = 0.5 * float(delta @ (lam * D * delta - g))
        P1 = apply_step(poses, delta, col)
        F1 = cost(P1, edges, deltas)
        gain = (F - F1) / L if L != 0.0 else float("nan")
        acc = ba.accept_step(L, F1, gain)
        trace.append(ba.IterRecord(F, F1, lam, gain, L, float(np.linalg.norm(delta)), acc, len(edges), len(edges),
                                   math.sqrt(2.0 * F / len(edges)), False, delta))
        lam, nu = ba.nielsen_update(lam, nu, gain, acc)
        if acc:
            poses, lin = P1, None
    return poses, lam, nu, trace
