"""Oracle for the loop-closure relative pose, one query frame at a time.

TEST INFRASTRUCTURE ONLY (like oracle/ba.py): only tests/, __graft_entry__.smoke() and
bench.py's CPU legs may use it.  It shares no code with the CUDA library.

What it computes (cuVSLAM, arXiv 2506.04359, Sec. 2.3, relative pose estimation): with
T^mw the pose of a map keyframe (world to map frame), the landmarks are shifted into the
map frame and the query frame's relative pose is
    T^bm = argmin  sum_j sum_k rho(|pi(T^cb_k T^bm T^mw p^w_j) - o_{j,k}|^2),
solved as the motion-only bundle adjustment of oracle/pnp.py on the shifted landmarks.
"""
from __future__ import annotations

import numpy as np

from . import pnp


def shift(T_mw: np.ndarray, lms: np.ndarray) -> np.ndarray:
    """p^m = R^mw p^w + t^mw for every landmark."""
    return np.asarray(lms, float) @ T_mw[:, :3].T + T_mw[:, 3]


def compose(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """[R | t] of A B for (3, 4) transforms."""
    out = np.empty((3, 4))
    out[:, :3] = A[:, :3] @ B[:, :3]
    out[:, 3] = A[:, :3] @ B[:, 3] + A[:, 3]
    return out


def inverse(A: np.ndarray) -> np.ndarray:
    out = np.empty((3, 4))
    out[:, :3] = A[:, :3].T
    out[:, 3] = -A[:, :3].T @ A[:, 3]
    return out


def solve_queries(batch, T_mw, T_bm0, iters: int | None = None, frames=None, lam0: float = 1e-4,
                  z_min: float = 1e-3):
    """Oracle relative poses of the selected query frames of a synth.FrameBatch (its frames'
    observations) with map poses T_mw (F, 3, 4) from initial guesses T_bm0: list of (T_bm, trace)."""
    iters = batch.iters if iters is None else iters
    out = []
    for f in (range(batch.F) if frames is None else frames):
        cam, lm, uv = batch.frame(f)
        w = pnp.frame_window(batch.rig.intr, batch.rig.T_cb, batch.lm, cam, lm, uv, batch.huber_delta, z_min)
        T, lam, nu, tr = pnp.lm_solve(w, T_bm0[f], shift(T_mw[f], batch.lm), iters, lam0)
        out.append((T, tr))
    return out
