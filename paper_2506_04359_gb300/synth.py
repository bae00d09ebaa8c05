"""Seeded synthetic sliding-window bundle-adjustment problems.

This module only *creates inputs*: a camera rig, a keyframe trajectory, landmarks,
their noisy pixel observations and a perturbed initial guess.  It holds none of the
solver's arithmetic (no residual Jacobians, no normal equations, no LM); the single
piece of geometry it shares with the method is the forward pinhole camera model used
to synthesise observations, written here independently in camera-centre form
(X_c = R_wc^T (p - c_wc)) rather than the solver's transform chain.

The problem statement follows cuVSLAM Sec. 2.2 (Eq. r^repr and the SBA objective):
keyframe poses T^bw_i (base-from-world), a rig of cameras with fixed camera-from-base
extrinsics T^cb_k, landmarks p^w_j, and observations o_{j,k} of landmark j by camera
k at keyframe i.  The multi-camera rig is a set of stereo pairs (Sec. 2.2,
"Multi-Stereo").

Random streams (numpy PCG64 via SeedSequence(seed).spawn) are drawn in a fixed order:
trajectory -> landmarks and tracks -> pixel noise -> outliers -> initial-guess
perturbation -> observation shuffle.  Each stream is independent, so changing one
stage never shifts another stage's draws.

Conventions: camera axes x right, y down, z forward; base frame = left camera frame of
stereo pair 0 for single-pair rigs; a pose is stored as a (3, 4) matrix [R | t] with
X_b = R X_w + t.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np
from scipy.spatial.transform import Rotation

__all__ = ["Rig", "Problem", "make_rig", "make_problem", "make_batch", "CONFIGS", "FrameBatch", "make_frames",
           "FRAME_CONFIGS"]


@dataclass
class Rig:
    intr: np.ndarray   # (C, 4) fx, fy, cx, cy
    T_cb: np.ndarray   # (C, 3, 4) camera-from-base [R | t]
    wh: np.ndarray     # (C, 2) image width, height (int)
    n_pairs: int

    @property
    def n_cams(self) -> int:
        return int(self.intr.shape[0])


@dataclass
class Problem:
    name: str
    seed: int
    rig: Rig
    poses_gt: np.ndarray    # (K, 3, 4) T^bw ground truth
    poses0: np.ndarray      # (K, 3, 4) initial guess
    lm_gt: np.ndarray       # (M, 3)
    lm0: np.ndarray         # (M, 3)
    obs_kf: np.ndarray      # (N,) int32
    obs_cam: np.ndarray     # (N,) int32
    obs_lm: np.ndarray      # (N,) int32
    obs_uv: np.ndarray      # (N, 2) float64
    outlier: np.ndarray     # (N,) bool
    fixed_kf: int = 0
    iters: int = 10
    huber_delta: float = 1.0
    precision: str = "fp64"
    info: dict = field(default_factory=dict)

    @property
    def K(self) -> int:
        return int(self.poses0.shape[0])

    @property
    def M(self) -> int:
        return int(self.lm0.shape[0])

    @property
    def N(self) -> int:
        return int(self.obs_kf.shape[0])

    @property
    def C(self) -> int:
        return self.rig.n_cams

    def copy(self) -> "Problem":
        return dataclasses.replace(
            self,
            poses_gt=self.poses_gt.copy(), poses0=self.poses0.copy(),
            lm_gt=self.lm_gt.copy(), lm0=self.lm0.copy(),
            obs_kf=self.obs_kf.copy(), obs_cam=self.obs_cam.copy(),
            obs_lm=self.obs_lm.copy(), obs_uv=self.obs_uv.copy(),
            outlier=self.outlier.copy(), info=dict(self.info))


# ----------------------------------------------------------------------------- rig

def _rot_y(a: float) -> np.ndarray:
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def make_rig(n_pairs: int, baseline: float, fx: float, fy: float, cx: float, cy: float,
             width: int, height: int, r_rig: float = 0.0) -> Rig:
    """Stereo pairs yawed by p*360/P about the base y axis (vertical, y down).

    The left camera of pair p sits r_rig metres along its own optical axis from the
    base origin; the right camera sits `baseline` metres along the left camera's x axis.
    """
    intr, T_cb, wh = [], [], []
    for p in range(n_pairs):
        R_bc = _rot_y(2.0 * np.pi * p / n_pairs)      # camera axes expressed in base
        c_left = r_rig * R_bc[:, 2]
        c_right = c_left + baseline * R_bc[:, 0]
        for c in (c_left, c_right):
            R = R_bc.T
            T_cb.append(np.concatenate([R, (-R @ c)[:, None]], axis=1))
            intr.append([fx, fy, cx, cy])
            wh.append([width, height])
    return Rig(np.array(intr, float), np.array(T_cb, float), np.array(wh, np.int64), n_pairs)


# ----------------------------------------------------------------------- trajectory

def _trajectory(kind: str, K: int, rng: np.random.Generator, **kw):
    """Base positions c_i (world) and yaw headings psi_i (rotation about world y)."""
    if kind == "line":                     # lateral motion along +x, looking +z
        step = kw.get("step", 0.5)
        c = np.stack([np.arange(K) * step, np.zeros(K), np.zeros(K)], 1)
        psi = np.zeros(K)
    elif kind == "arc":                    # start at origin heading +z, turn right
        length, angle = kw["length"], kw["angle"]
        r = length / angle
        th = np.linspace(0.0, angle, K)
        c = np.stack([r - r * np.cos(th), np.zeros(K), r * np.sin(th)], 1)
        psi = th                           # tangent (sin th, 0, cos th)
    elif kind == "circle":                 # closed loop, heading tangent
        radius = kw["radius"]
        th = 2.0 * np.pi * np.arange(K) / K
        c = np.stack([radius * np.sin(th), np.zeros(K), -radius * np.cos(th)], 1)
        c = c - c[0]
        psi = np.arctan2(np.cos(th), np.sin(th))   # tangent (cos th, 0, sin th)
    elif kind == "randwalk":               # persistent-heading planar random walk
        step, turn = kw["step"], kw["turn_sigma"]
        psi = np.zeros(K)
        c = np.zeros((K, 3))
        turns = rng.normal(0.0, turn, K)
        for i in range(1, K):
            psi[i] = psi[i - 1] + turns[i]
            c[i] = c[i - 1] + step * np.array([np.sin(psi[i]), 0.0, np.cos(psi[i])])
    else:
        raise ValueError(kind)
    R_wb = np.stack([_rot_y(a) for a in psi])          # base axes in world
    return c, R_wb


def _poses_from(c: np.ndarray, R_wb: np.ndarray) -> np.ndarray:
    R = np.transpose(R_wb, (0, 2, 1))
    t = -np.einsum("kij,kj->ki", R, c)
    return np.concatenate([R, t[:, :, None]], axis=2)


# -------------------------------------------------------------------- observations

def _camera_frames(rig: Rig, c_w: np.ndarray, R_wb: np.ndarray):
    """World rotation R_wc (K, C, 3, 3) and centre c_wc (K, C, 3) of every camera."""
    R_bc = np.transpose(rig.T_cb[:, :, :3], (0, 2, 1))            # (C,3,3)
    c_bc = -np.einsum("cij,ci->cj", rig.T_cb[:, :, :3], rig.T_cb[:, :, 3])  # R^T(-t)
    R_wc = np.einsum("kij,cjl->kcil", R_wb, R_bc)
    c_wc = c_w[:, None, :] + np.einsum("kij,cj->kci", R_wb, c_bc)
    return R_wc, c_wc


def _observe_chunk(rig, R_wb, c_w, R_wc, c_wc, pts, near, far):
    """Pixel coordinates and visibility of pts (B,3) in the two cameras of the stereo
    pair whose optical axis is closest to the point's direction, at every keyframe.

    Returns u, v, vis of shape (B, K, 2) and the camera index of each slot (B, K, 2)."""
    d_b = np.einsum("kji,bkj->bki", R_wb, pts[:, None, :] - c_w[None])   # R_wb^T (p - c)
    axes = np.stack([rig.T_cb[2 * q, 2, :3] for q in range(rig.n_pairs)])  # optical axes in base
    best = np.argmax(np.einsum("bki,pi->bkp", d_b, axes), axis=2)         # (B,K)
    cam = np.stack([2 * best, 2 * best + 1], axis=2)                       # (B,K,2)
    kk = np.broadcast_to(np.arange(R_wb.shape[0])[None, :, None], cam.shape)
    Rg = R_wc[kk, cam]                                                     # (B,K,2,3,3)
    d = pts[:, None, None, :] - c_wc[kk, cam]                              # (B,K,2,3)
    Xc = np.einsum("bksji,bksj->bksi", Rg, d)                              # R_wc^T d
    Z = Xc[..., 2]
    intr = rig.intr[cam]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = intr[..., 0] * Xc[..., 0] / Z + intr[..., 2]
        v = intr[..., 1] * Xc[..., 1] / Z + intr[..., 3]
    wh = rig.wh[cam]
    vis = (Z > near) & (u >= 0) & (u < wh[..., 0]) & (v >= 0) & (v < wh[..., 1])
    if far is not None:
        vis &= np.linalg.norm(d, axis=-1) <= far
    return u, v, vis, cam


# ------------------------------------------------------------------------ configs

# Each config restates a workload: rig, trajectory, landmark volume, visibility rule,
# noise, outliers, perturbation and solve settings.  "track" gives the range of track
# lengths (consecutive keyframes) over which one landmark is observed; None means every
# keyframe that sees it.  Volumes are axis-aligned boxes (lo, hi) in world coordinates
# or a cylinder around the trajectory's loop centre.
CONFIGS = {
    "c0": dict(
        rig=dict(n_pairs=1, baseline=0.12, fx=458.0, fy=458.0, cx=367.0, cy=248.0, width=752, height=480),
        traj=dict(kind="line", K=5, step=0.5),
        volume=dict(kind="box", lo=(-4.0, -2.0, 2.0), hi=(4.0, 2.0, 10.0)),
        M=400, track=None, near=0.5, far=None,
        sigma=0.5, outlier_frac=0.0, iters=10, huber=1.0, precision="fp64"),
    "c1": dict(
        rig=dict(n_pairs=1, baseline=0.12, fx=458.0, fy=458.0, cx=367.0, cy=248.0, width=752, height=480),
        traj=dict(kind="arc", K=20, length=10.0, angle=np.pi / 2),
        volume=dict(kind="box", lo=(-4.0, -2.0, 8.5), hi=(16.0, 2.0, 16.5)),
        M=5000, track=(5, 12), near=0.5, far=None,
        sigma=0.5, outlier_frac=0.05, iters=20, huber=1.0, precision="mixed"),
    "c2": dict(
        rig=dict(n_pairs=4, baseline=0.12, fx=458.0, fy=458.0, cx=367.0, cy=248.0, width=752, height=480, r_rig=0.15),
        traj=dict(kind="circle", K=50, radius=5.0),
        volume=dict(kind="cylinder", r_lo=8.0, r_hi=12.0, y_lo=-2.0, y_hi=2.0),
        M=20000, track=(4, 14), near=0.5, far=None,
        sigma=0.5, outlier_frac=0.0, iters=10, huber=1.0, precision="mixed"),
    "c4": dict(
        rig=dict(n_pairs=16, baseline=0.1, fx=320.0, fy=320.0, cx=320.0, cy=240.0, width=640, height=480, r_rig=0.15),
        traj=dict(kind="randwalk", K=100, step=0.5, turn_sigma=0.35),
        volume=dict(kind="box_around", half=(30.0, 3.0, 30.0)),
        M=200000, track=(5, 20), near=0.5, far=20.0,
        sigma=0.7, outlier_frac=0.03, iters=15, huber=1.0, precision="mixed"),
}


def _sample_volume(vol: dict, n: int, rng: np.random.Generator, c_w: np.ndarray):
    if vol["kind"] == "box":
        lo, hi = np.array(vol["lo"]), np.array(vol["hi"])
        return lo + (hi - lo) * rng.random((n, 3))
    if vol["kind"] == "box_around":
        centre = 0.5 * (c_w.min(0) + c_w.max(0))
        half = np.array(vol["half"])
        return centre - half + 2.0 * half * rng.random((n, 3))
    if vol["kind"] == "cylinder":
        centre = c_w.mean(0)
        r = np.sqrt(vol["r_lo"] ** 2 + (vol["r_hi"] ** 2 - vol["r_lo"] ** 2) * rng.random(n))
        a = 2.0 * np.pi * rng.random(n)
        y = vol["y_lo"] + (vol["y_hi"] - vol["y_lo"]) * rng.random(n)
        return np.stack([centre[0] + r * np.cos(a), y, centre[2] + r * np.sin(a)], 1)
    raise ValueError(vol["kind"])


def _generate(name: str, seed: int, cfg: dict) -> Problem:
    ss = np.random.SeedSequence(seed)
    r_traj, r_lm, r_noise, r_out, r_pert, r_shuf = [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(6)]

    rig = make_rig(**cfg["rig"])
    tr = dict(cfg["traj"])
    K = tr.pop("K")
    c_w, R_wb = _trajectory(tr.pop("kind"), K, r_traj, **tr)
    poses_gt = _poses_from(c_w, R_wb)
    R_wc, c_wc = _camera_frames(rig, c_w, R_wb)

    M_target = cfg["M"]
    lms, obs = [], []        # obs rows: (lm, kf, cam, u, v)
    n_acc = 0
    chunk = int(max(256, min(8192, 4_000_000 // (K * 2))))
    tries = 0
    while n_acc < M_target:
        tries += 1
        if tries > 4000:
            raise RuntimeError(f"{name}: could not place {M_target} visible landmarks")
        pts = _sample_volume(cfg["volume"], chunk, r_lm, c_w)
        u, v, vis, cam = _observe_chunk(rig, R_wb, c_w, R_wc, c_wc, pts, cfg["near"], cfg["far"])
        # track window over consecutive keyframes, starting at a keyframe that sees the point
        kf_vis = vis.any(axis=2)                                   # (B,K)
        u_start = r_lm.random(chunk)
        if cfg["track"] is not None:
            lo, hi = cfg["track"]
            L = r_lm.integers(lo, hi + 1, chunk)
            nv = kf_vis.sum(1)
            pick = np.minimum((u_start * nv).astype(np.int64), np.maximum(nv - 1, 0))
            csum = np.cumsum(kf_vis, axis=1) - 1                   # rank among visible kfs
            start = np.argmax((csum == pick[:, None]) & kf_vis, axis=1)
            kk = np.arange(K)[None, :]
            win = (kk >= start[:, None]) & (kk < (start + L)[:, None])
            vis &= win[:, :, None]
        cnt = vis.reshape(chunk, -1).sum(1)
        ok = np.nonzero(cnt >= 2)[0]
        ok = ok[: M_target - n_acc]
        if ok.size:
            bb, kfs, slot = np.nonzero(vis[ok])          # sorted by landmark, keyframe, camera
            src = ok[bb]
            cams = cam[src, kfs, slot]
            obs.append(np.stack([n_acc + bb, kfs, cams, u[src, kfs, slot], v[src, kfs, slot]], 1))
            lms.append(pts[ok])
            n_acc += ok.size
    lm_gt = np.concatenate(lms, 0)
    O = np.concatenate(obs, 0)
    obs_lm = O[:, 0].astype(np.int32)
    obs_kf = O[:, 1].astype(np.int32)
    obs_cam = O[:, 2].astype(np.int32)
    uv = O[:, 3:5].copy()
    N = uv.shape[0]

    # pixel noise, then outliers (uniform over the image)
    uv += r_noise.normal(0.0, cfg["sigma"], (N, 2)) if cfg["sigma"] > 0 else 0.0
    outlier = r_out.random(N) < cfg["outlier_frac"]
    n_out = int(outlier.sum())
    if n_out:
        wh = rig.wh[obs_cam[outlier]]
        uv[outlier] = r_out.random((n_out, 2)) * wh

    poses0, lm0 = perturb(poses_gt, lm_gt, r_pert, fixed_kf=0,
                          sigma_t=0.05, sigma_r_deg=1.0, sigma_l=0.10)

    perm = r_shuf.permutation(N)
    obs_kf, obs_cam, obs_lm, uv, outlier = obs_kf[perm], obs_cam[perm], obs_lm[perm], uv[perm], outlier[perm]

    pairs = np.unique(obs_lm.astype(np.int64) * K + obs_kf).size
    info = dict(K=K, C=rig.n_cams, M=int(lm_gt.shape[0]), N=int(N), n_outlier=n_out, n_pairs=int(pairs),
                n_c=6 * (K - 1), n_f=6 * (K - 1) + 3 * int(lm_gt.shape[0]))
    return Problem(name=name, seed=seed, rig=rig, poses_gt=poses_gt, poses0=poses0, lm_gt=lm_gt, lm0=lm0,
                   obs_kf=np.ascontiguousarray(obs_kf), obs_cam=np.ascontiguousarray(obs_cam),
                   obs_lm=np.ascontiguousarray(obs_lm), obs_uv=np.ascontiguousarray(uv),
                   outlier=outlier, fixed_kf=0, iters=cfg["iters"], huber_delta=cfg["huber"],
                   precision=cfg["precision"], info=info)


def perturb(poses: np.ndarray, lms: np.ndarray, rng: np.random.Generator, fixed_kf: int = 0,
            sigma_t: float = 0.05, sigma_r_deg: float = 1.0, sigma_l: float = 0.10):
    """Initial guess: left rotation noise Exp(phi), phi ~ N(0, sigma_r^2 I); translation and
    landmark noise per axis.  The gauge keyframe is left at its true value."""
    K, M = poses.shape[0], lms.shape[0]
    phi = rng.normal(0.0, np.deg2rad(sigma_r_deg), (K, 3))
    dt = rng.normal(0.0, sigma_t, (K, 3))
    dl = rng.normal(0.0, sigma_l, (M, 3))
    out = poses.copy()
    Rn = Rotation.from_rotvec(phi).as_matrix()
    for i in range(K):
        if i == fixed_kf:
            continue
        out[i, :, :3] = Rn[i] @ poses[i, :, :3]
        out[i, :, 3] = poses[i, :, 3] + dt[i]
    return out, lms + dl


def make_problem(name: str = "c0", seed: int = 0, **overrides) -> Problem:
    """Build one named workload.  `overrides` replace top-level config keys (for tests:
    e.g. sigma=0, outlier_frac=0, M=50)."""
    if name not in CONFIGS:
        raise KeyError(name)
    cfg = dict(CONFIGS[name])
    for k, v in overrides.items():
        if k in ("K",):
            cfg["traj"] = dict(cfg["traj"], K=v)
        else:
            cfg[k] = v
    return _generate(name, seed, cfg)


def c3_window_config(seed: int) -> dict:
    """Per-window settings of the batched workload: K ~ U[5,30], M ~ U[300,3000],
    a rig of {1,2,4,8} stereo pairs; noise and perturbation as the small stereo case."""
    r = np.random.Generator(np.random.PCG64(np.random.SeedSequence([3, seed])))
    K = int(r.integers(5, 31))
    M = int(r.integers(300, 3001))
    P = int(r.choice([1, 2, 4, 8]))
    rig = dict(n_pairs=P, baseline=0.12, fx=458.0, fy=458.0, cx=367.0, cy=248.0, width=752, height=480,
               r_rig=0.0 if P == 1 else 0.15)
    if P == 1:
        vol = dict(kind="box", lo=(-4.0, -2.0, 2.0), hi=(0.5 * (K - 1) + 4.0, 2.0, 10.0))
        traj = dict(kind="line", K=K, step=0.5)
    else:
        vol = dict(kind="cylinder", r_lo=6.0, r_hi=10.0, y_lo=-2.0, y_hi=2.0)
        traj = dict(kind="circle", K=K, radius=3.0)
    return dict(rig=rig, traj=traj, volume=vol, M=M, track=(3, 8), near=0.5, far=None,
                sigma=0.5, outlier_frac=0.0, iters=10, huber=1.0, precision="mixed")


def make_batch(n_windows: int = 256, first_seed: int = 0) -> list[Problem]:
    """Independent BA windows of uneven size (the batched workload), seeds first_seed..."""
    return [_generate(f"c3w{s}", s, c3_window_config(s)) for s in range(first_seed, first_seed + n_windows)]


# ------------------------------------------------------------- frames (motion-only BA)

@dataclass
class FrameBatch:
    """Independent frames for motion-only bundle adjustment (multi-camera PnP): each frame
    has one base pose and observations of fixed map landmarks.  Observations are grouped by
    frame: those of frame f are [frame_off[f], frame_off[f + 1])."""
    name: str
    seed: int
    rig: Rig
    poses_gt: np.ndarray    # (F, 3, 4) T^bw ground truth
    poses0: np.ndarray      # (F, 3, 4) initial guess
    lm: np.ndarray          # (M, 3) map landmarks (held fixed)
    frame_off: np.ndarray   # (F + 1,) int32
    obs_cam: np.ndarray     # (N,) int32
    obs_lm: np.ndarray      # (N,) int32
    obs_uv: np.ndarray      # (N, 2)
    outlier: np.ndarray     # (N,) bool
    iters: int = 10
    huber_delta: float = 1.0

    @property
    def F(self) -> int:
        return int(self.poses0.shape[0])

    @property
    def N(self) -> int:
        return int(self.obs_cam.shape[0])

    @property
    def M(self) -> int:
        return int(self.lm.shape[0])

    @property
    def C(self) -> int:
        return self.rig.n_cams

    def frame(self, f: int):
        """(cam, lm, uv) of frame f."""
        a, b = int(self.frame_off[f]), int(self.frame_off[f + 1])
        return self.obs_cam[a:b], self.obs_lm[a:b], self.obs_uv[a:b]


FRAME_CONFIGS = {
    # stereo tracking frames: the small stereo rig, 300 map points per frame
    "pnp_stereo": dict(rig=CONFIGS["c0"]["rig"], frames=1024, lm_per_frame=300, depth=(2.0, 12.0),
                       sigma=0.5, outlier_frac=0.05, iters=10),
    # multi-camera tracking frames: the 16-pair ring, ~400 map points per frame, each seen by
    # about eight of the 32 cameras
    "pnp_multi": dict(rig=CONFIGS["c4"]["rig"], frames=512, lm_per_frame=400, depth=(1.0, 15.0),
                      sigma=0.7, outlier_frac=0.03, iters=10),
}


def make_frames(name: str = "pnp_stereo", seed: int = 0, **overrides) -> FrameBatch:
    """Frames at random base poses (position in a 40 m square, heading uniform).  Each map
    point is placed by choosing a camera, a pixel uniform over its image and a depth uniform
    in `depth`, and is then observed by every camera of the rig in whose image it falls
    (depth > 0.5 m).  Pixel noise, uniform outliers and the initial-guess perturbation (5 cm,
    1 deg) as for the windows.  Draw order: poses -> points -> noise -> outliers ->
    perturbation."""
    cfg = dict(FRAME_CONFIGS[name])
    cfg.update(overrides)
    ss = np.random.SeedSequence([7, seed])
    r_pose, r_pts, r_noise, r_out, r_pert = [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(5)]
    rig = make_rig(**cfg["rig"])
    F, Mf = cfg["frames"], cfg["lm_per_frame"]
    c_w = np.stack([r_pose.uniform(-20, 20, F), r_pose.uniform(-0.5, 0.5, F), r_pose.uniform(-20, 20, F)], 1)
    R_wb = np.stack([_rot_y(a) for a in r_pose.uniform(-np.pi, np.pi, F)])
    poses_gt = _poses_from(c_w, R_wb)
    R_wc, c_wc = _camera_frames(rig, c_w, R_wb)                         # (F,C,3,3), (F,C,3)
    C = rig.n_cams
    cam0 = r_pts.integers(0, C, (F, Mf))
    wh = rig.wh[cam0].astype(np.float64)
    px = r_pts.random((F, Mf, 2)) * wh
    depth = r_pts.uniform(cfg["depth"][0], cfg["depth"][1], (F, Mf))
    intr0 = rig.intr[cam0]
    ray = np.stack([(px[..., 0] - intr0[..., 2]) / intr0[..., 0], (px[..., 1] - intr0[..., 3]) / intr0[..., 1],
                    np.ones((F, Mf))], -1) * depth[..., None]
    ff = np.arange(F)[:, None]
    pts = np.einsum("fmij,fmj->fmi", R_wc[ff, cam0], ray) + c_wc[ff, cam0]   # (F,Mf,3)
    # project into every camera
    d = pts[:, :, None, :] - c_wc[:, None, :, :]                           # (F,Mf,C,3)
    Xc = np.einsum("fcji,fmcj->fmci", R_wc, d)
    Z = Xc[..., 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = rig.intr[:, 0] * Xc[..., 0] / Z + rig.intr[:, 2]
        v = rig.intr[:, 1] * Xc[..., 1] / Z + rig.intr[:, 3]
    vis = (Z > 0.5) & (u >= 0) & (u < rig.wh[:, 0]) & (v >= 0) & (v < rig.wh[:, 1])
    fi, mi, ci = np.nonzero(vis)                                            # sorted by frame
    obs_lm = (fi * Mf + mi).astype(np.int32)
    obs_cam = ci.astype(np.int32)
    uv = np.stack([u[fi, mi, ci], v[fi, mi, ci]], 1)
    N = uv.shape[0]
    uv += r_noise.normal(0.0, cfg["sigma"], (N, 2))
    outlier = r_out.random(N) < cfg["outlier_frac"]
    n_out = int(outlier.sum())
    if n_out:
        uv[outlier] = r_out.random((n_out, 2)) * rig.wh[obs_cam[outlier]]
    poses0, _ = perturb(poses_gt, np.zeros((0, 3)), r_pert, fixed_kf=-1, sigma_t=0.05, sigma_r_deg=1.0,
                        sigma_l=0.0)
    frame_off = np.concatenate([[0], np.cumsum(np.bincount(fi, minlength=F))]).astype(np.int32)
    return FrameBatch(name=name, seed=seed, rig=rig, poses_gt=poses_gt, poses0=poses0, lm=pts.reshape(-1, 3),
                      frame_off=frame_off, obs_cam=obs_cam, obs_lm=obs_lm, obs_uv=np.ascontiguousarray(uv),
                      outlier=outlier, iters=cfg["iters"], huber_delta=1.0)


def landmark_segments(obs_lm: np.ndarray, M: int):
    """Observations grouped by landmark (stable): the permutation `order` and the segment
    offsets lm_off (M + 1) with the observations of landmark j at order[lm_off[j]:lm_off[j+1]]."""
    obs_lm = np.asarray(obs_lm, np.int64)
    order = np.argsort(obs_lm, kind="stable").astype(np.int64)
    lm_off = np.concatenate([[0], np.cumsum(np.bincount(obs_lm, minlength=M))]).astype(np.int32)
    return order, lm_off


def make_map_poses(batch: FrameBatch, seed: int = 0, sigma_r_deg: float = 20.0, sigma_t: float = 5.0):
    """Loop-closure queries on a frame batch: a map keyframe pose T^mw per frame (world to map
    frame: rotation N(0, sigma_r) about a random axis, translation N(0, sigma_t) per axis) and
    the initial relative pose T^bm0 = T^bw0 (T^mw)^-1 from the frame's initial guess.
    Returns (T_mw, T_bm0), each (F, 3, 4)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([11, seed])))
    F = batch.F
    R = Rotation.from_rotvec(rng.normal(0.0, np.deg2rad(sigma_r_deg), (F, 3))).as_matrix()
    t = rng.normal(0.0, sigma_t, (F, 3))
    T_mw = np.concatenate([R, t[:, :, None]], axis=2)
    Rinv = np.transpose(R, (0, 2, 1))
    tinv = -np.einsum("fij,fj->fi", Rinv, t)
    T_bm0 = np.empty((F, 3, 4))
    T_bm0[:, :, :3] = np.einsum("fij,fjk->fik", batch.poses0[:, :, :3], Rinv)
    T_bm0[:, :, 3] = np.einsum("fij,fj->fi", batch.poses0[:, :, :3], tinv) + batch.poses0[:, :, 3]
    return T_mw, T_bm0


# ------------------------------------------------------------------------ pose graphs

@dataclass
class PoseGraph:
    """A pose graph: world-from-base keyframe poses and relative-pose edges (i, j) with
    measured deltas D_ij ~ T_i^-1 T_j.  Pose `fixed` is the gauge."""
    name: str
    seed: int
    poses_gt: np.ndarray    # (K, 3, 4) world-from-base
    poses0: np.ndarray      # (K, 3, 4) initial guess (dead reckoning along the odometry chain)
    edges: np.ndarray       # (E, 2) int32
    deltas: np.ndarray      # (E, 3, 4)
    fixed: int = 0
    iters: int = 10

    @property
    def K(self) -> int:
        return int(self.poses0.shape[0])

    @property
    def E(self) -> int:
        return int(self.edges.shape[0])


def _compose(A, B):
    out = np.empty((3, 4))
    out[:, :3] = A[:, :3] @ B[:, :3]
    out[:, 3] = A[:, :3] @ B[:, 3] + A[:, 3]
    return out


def _inverse(A):
    out = np.empty((3, 4))
    out[:, :3] = A[:, :3].T
    out[:, 3] = -A[:, :3].T @ A[:, 3]
    return out


def _exp_noise(rng, sigma_t, sigma_r_deg):
    """A small random transform: rotation Exp(phi), phi ~ N(0, sigma_r^2 I), translation N(0, sigma_t^2 I)."""
    out = np.empty((3, 4))
    out[:, :3] = Rotation.from_rotvec(rng.normal(0.0, np.deg2rad(sigma_r_deg), 3)).as_matrix()
    out[:, 3] = rng.normal(0.0, sigma_t, 3)
    return out


PGO_CONFIGS = {
    # two laps of a 10 m circle (with a slow vertical wave), odometry between consecutive
    # keyframes, loop closures from every fifth keyframe of the first lap to the second
    "pgo_loop": dict(K=200, laps=2, radius=10.0, odo=(0.02, 0.2), loop=(0.01, 0.1), loop_every=5, iters=10),
    # a longer map: four laps, 600 keyframes
    "pgo_large": dict(K=600, laps=4, radius=15.0, odo=(0.02, 0.2), loop=(0.01, 0.1), loop_every=5, iters=10),
}


def make_pose_graph(name: str = "pgo_loop", seed: int = 0, **overrides) -> PoseGraph:
    """Draw order: odometry noise -> loop-closure noise (independent streams)."""
    cfg = dict(PGO_CONFIGS[name])
    cfg.update(overrides)
    ss = np.random.SeedSequence([13, seed])
    r_odo, r_loop = [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(2)]
    K, laps, rad = cfg["K"], cfg["laps"], cfg["radius"]
    th = 2.0 * np.pi * laps * np.arange(K) / K
    poses = np.empty((K, 3, 4))
    for k in range(K):
        R = Rotation.from_euler("yxz", [th[k] + np.pi / 2, 0.05 * np.sin(3 * th[k]), 0.0]).as_matrix()
        poses[k, :, :3] = R
        poses[k, :, 3] = [rad * np.cos(th[k]), 0.3 * np.sin(th[k] / laps), rad * np.sin(th[k])]
    edges, deltas = [], []
    for k in range(K - 1):
        edges.append((k, k + 1))
        deltas.append(_compose(_compose(_inverse(poses[k]), poses[k + 1]), _exp_noise(r_odo, *cfg["odo"])))
    per_lap = K // laps
    for k in (range(0, K - per_lap, cfg["loop_every"]) if cfg["loop_every"] > 0 else []):
        j = k + per_lap
        edges.append((k, j))
        deltas.append(_compose(_compose(_inverse(poses[k]), poses[j]), _exp_noise(r_loop, *cfg["loop"])))
    poses0 = np.empty_like(poses)
    poses0[0] = poses[0]
    for k in range(K - 1):
        poses0[k + 1] = _compose(poses0[k], deltas[k])
    return PoseGraph(name=name, seed=seed, poses_gt=poses, poses0=poses0, edges=np.array(edges, np.int32),
                     deltas=np.array(deltas), fixed=0, iters=cfg["iters"])
