"""The host layer's tables on the CPU: cvba_host.cpp compiled into a driver over a stand-in for
the CUDA runtime (device memory is host memory, the kernel launchers do nothing), a window
loaded through the C ABI, and every table the kernels receive checked against its definition:

* slot-order pixels and cameras, the (landmark, keyframe) pairs and their offsets, each
  landmark's off-diagonal block offsets (m(m-1)/2 for m pairs), the free-keyframe map;
* linearisation tiles: a partition of the internal landmarks into runs, each within the pair
  and landmark limits and maximal (the next landmark would break one), with its pair,
  observation and keyframe ranges; per tile and keyframe the tile-local free pairs in pair
  order; per keyframe its partial slots in tile order;
* Schur tiles (landmarks sharing one window of at most SPAN_MAX free keyframes) and direct
  tiles (wider landmarks): together a partition, each maximal, with window partial offsets;
  per block of the reduced camera system the covering tiles' partial offsets; the blocks the
  reduction writes;
* the factor's envelope per 32-column panel;
* rig, poses and landmarks (internal order) in the device layouts, FP32 mirrors, the buffers
  that start at zero, the control block;
* poses and landmarks replaced after the layout (only that half written), and read back.

The driver runs under AddressSanitizer where the compiler has it, with the pinned staging
allocated at exactly the size the layout asks for, so an overrun of the staging fails here."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import ba
from paper_2506_04359_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2506_04359_gb300", "csrc")
N_SM = 152


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not cxx or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    out = str(tmp_path_factory.mktemp("drv") / "host_tables_driver")
    base = [cxx, "-O1", "-g", "-std=c++17", "-pthread", "-I", cuda_inc, "-I", CSRC,
            os.path.join(ROOT, "tests", "host_tables_driver.cpp"), os.path.join(CSRC, "cvba_layout.cpp"), "-o", out]
    r = subprocess.run(base[:1] + ["-fsanitize=address"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:                    # no sanitizer runtime: plain build
        subprocess.run(base, check=True, capture_output=True)
    return out


class Window:
    """Observations and state of one window, written for the driver."""

    def __init__(self, K, C, M, fixed, kf, cam, lm, uv, intr, T_cb, poses, lms, seed=0):
        self.K, self.C, self.M, self.fixed = K, C, M, fixed
        self.kf, self.cam, self.lm = (np.asarray(a, np.int32) for a in (kf, cam, lm))
        self.N = len(self.kf)
        self.uv = np.asarray(uv, np.float64).reshape(self.N, 2)
        self.intr, self.T_cb = np.asarray(intr, np.float64), np.asarray(T_cb, np.float64).reshape(C, 3, 4)
        self.poses, self.lms = np.asarray(poses, np.float64).reshape(K, 3, 4), np.asarray(lms, np.float64).reshape(M, 3)
        rng = np.random.default_rng(seed + 99)
        self.poses2 = self.poses + rng.normal(0, 1e-3, self.poses.shape)
        self.lms2 = self.lms + rng.normal(0, 1e-2, self.lms.shape)

    @classmethod
    def from_problem(cls, p):
        return cls(p.K, p.C, p.M, p.fixed_kf, p.obs_kf, p.obs_cam, p.obs_lm, p.obs_uv, p.rig.intr, p.rig.T_cb,
                   p.poses0, p.lm0)

    def write(self, d):
        with open(os.path.join(d, "dims.txt"), "w") as f:
            f.write(f"{self.K} {self.C} {self.M} {self.N} {self.fixed}")
        for name, a in (("kf", self.kf), ("cam", self.cam), ("lm", self.lm), ("uv", self.uv), ("intr", self.intr),
                        ("tcb", self.T_cb), ("poses", self.poses), ("lms", self.lms), ("poses2", self.poses2),
                        ("lms2", self.lms2)):
            np.ascontiguousarray(a).tofile(os.path.join(d, f"{name}.bin"))


def wide_window(seed=0):
    """30 keyframes, 2 cameras: most landmarks seen from a few consecutive keyframes, some
    from keyframes spread over the whole window (wider than a Schur tile's window), the fixed
    keyframe in the middle."""
    rng = np.random.default_rng(seed)
    K, C, M = 30, 2, 3000
    kf, cam, lm = [], [], []
    for j in range(M):
        if rng.random() < 0.05:
            ks = rng.choice(K, size=rng.integers(24, K + 1), replace=False)
        else:
            a = rng.integers(0, K - 3)
            ks = np.arange(a, a + rng.integers(2, 5))
        for k in ks:
            for c in range(C):
                if c == 0 or rng.random() < 0.5:
                    kf.append(k), cam.append(c), lm.append(j)
    kf[:K] = list(range(K))                  # every keyframe observed (landmarks keep >= 2 views)
    perm = rng.permutation(len(kf))
    kf, cam, lm = (np.asarray(a)[perm] for a in (kf, cam, lm))
    N = len(kf)
    intr = np.tile([400.0, 400.0, 320.0, 240.0], (C, 1))
    T_cb = np.tile(np.hstack([np.eye(3), np.zeros((3, 1))]), (C, 1, 1))
    poses = np.tile(np.hstack([np.eye(3), np.zeros((3, 1))]), (K, 1, 1))
    poses[:, :, 3] = rng.normal(0, 1, (K, 3))
    return Window(K, C, M, 12, kf, cam, lm, rng.normal(300, 50, (N, 2)), intr, T_cb, poses, rng.normal(0, 5, (M, 3)),
                  seed)


def small_window(K, C, M, fixed, seed=0):
    """A small random window: every landmark seen from 2 to 4 random (keyframe, camera) views,
    every keyframe observed."""
    rng = np.random.default_rng(seed)
    kf, cam, lm = [], [], []
    for j in range(M):
        for _ in range(rng.integers(2, 5)):
            kf.append(rng.integers(0, K)), cam.append(rng.integers(0, C)), lm.append(j)
    kf[:K] = list(range(K))
    N = len(kf)
    intr = np.tile([300.0, 310.0, 160.0, 120.0], (C, 1))
    T_cb = np.tile(np.hstack([np.eye(3), np.ones((3, 1))]), (C, 1, 1))
    poses = np.tile(np.hstack([np.eye(3), np.zeros((3, 1))]), (K, 1, 1))
    return Window(K, C, M, fixed, kf, cam, lm, rng.normal(100, 10, (N, 2)), intr, T_cb, poses,
                  rng.normal(0, 3, (M, 3)), seed)


def run(driver, d, w, prec, lin_pairs=0, schur_lms=0, chol_mode=0):
    w.write(d)
    r = subprocess.run([driver, d, prec, str(lin_pairs), str(schur_lms), str(chol_mode)], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    vals = [int(x) for x in open(os.path.join(d, "t_sizes.txt")).read().split()]
    keys = ["P", "n_c", "n_blk", "npw", "chol_blocked", "max_span", "max_panels", "LIN_TILE_PAIRS", "LIN_TILE_LMS",
            "SCHUR_TILE_PAIRS", "SCHUR_TILE_LMS", "SPAN_MAX", "RIG_STRIDE", "POSE_STRIDE"]
    sz = dict(zip(keys, vals))

    def t(name, dtype=np.int32):
        return np.fromfile(os.path.join(d, f"t_{name}.bin"), dtype)
    return sz, t


def check_tables(w, sz, t, prec, lin_pairs, schur_lms, chol_mode):
    K, C, M, N, fixed = w.K, w.C, w.M, w.N, w.fixed
    f64 = np.float64
    # --- layout and the arrays derived from it
    lo, oo, off = ba.device_layout(w.kf, w.cam, w.lm, M)
    assert np.array_equal(t("lm_order"), lo) and np.array_equal(t("obs_order"), oo)
    assert np.array_equal(t("d_lm_order"), lo)
    rank = np.empty(M, np.int64)
    rank[lo] = np.arange(M)
    if prec == "mixed":
        assert np.array_equal(t("obs_uv", np.float32).reshape(N, 2), w.uv[oo].astype(np.float32))
    else:
        assert np.array_equal(t("obs_uv", f64).reshape(N, 2), w.uv[oo])
    assert np.array_equal(t("obs_cam"), w.cam[oo])
    r_s, k_s = rank[w.lm[oo]], w.kf[oo]
    start = np.ones(N, bool)
    start[1:] = (r_s[1:] != r_s[:-1]) | (k_s[1:] != k_s[:-1])
    s = np.nonzero(start)[0]
    P = len(s)
    assert sz["P"] == P
    pk, pl = t("pair_kf"), t("pair_lm")
    assert np.array_equal(pk, k_s[s]) and np.array_equal(pl, r_s[s])
    po = t("pair_obs")
    assert np.array_equal(po, np.append(s, N))
    lp = t("lm_pair")
    assert np.array_equal(lp, np.searchsorted(pl, np.arange(M + 1), side="left"))
    m = np.diff(lp).astype(np.int64)
    lb = t("lm_blk")
    assert np.array_equal(lb, np.concatenate([[0], np.cumsum(m * (m - 1) // 2)]))
    kf_pb = t("kf_pb")
    assert np.array_equal(kf_pb, [-1 if a == fixed else (a if a < fixed else a - 1) for a in range(K)])
    free = kf_pb >= 0

    # --- linearisation tiles: a partition into maximal runs within the limits
    target = (min(sz["LIN_TILE_PAIRS"], lin_pairs) if lin_pairs > 0
              else max(32, min(sz["LIN_TILE_PAIRS"], math.ceil(P / (2 * N_SM)))))
    lt = t("lin_tiles").reshape(-1, 12)
    l0, l1, p0, p1, kflo, kfn, part, kfl_off, o0, o1, kfi0, kfi_n = lt.T
    assert l0[0] == 0 and l1[-1] == M and np.array_equal(l0[1:], l1[:-1]) and np.all(l1 > l0)
    npairs = lp[l1] - lp[l0]
    assert np.all((npairs <= target) | (l1 - l0 == 1)) and np.all(l1 - l0 <= sz["LIN_TILE_LMS"])
    nxt = l1[:-1]                                  # the next landmark would break a limit
    assert np.all((lp[nxt + 1] - lp[l0[:-1]] > target) | (l1[:-1] - l0[:-1] >= sz["LIN_TILE_LMS"]))
    assert np.array_equal(p0, lp[l0]) and np.array_equal(p1, lp[l1])
    assert np.array_equal(o0, po[p0]) and np.array_equal(o1, po[p1]) and np.all(part == -1)
    kmin = np.minimum.reduceat(pk, p0)
    kmax = np.maximum.reduceat(pk, p0)
    assert np.array_equal(kflo, kmin) and np.array_equal(kfn, kmax - kmin + 1)
    assert kfl_off[0] == 0 and np.array_equal(kfl_off[1:], np.cumsum(kfn + 1)[:-1])
    lko, lks, lki = t("lin_kf_off"), t("lin_kf_slot"), t("lin_kf_idx")
    kto = t("kf_tiles_off")
    cover = np.zeros(K, np.int64)
    for a in range(K):
        cover[a] = np.sum((kflo <= a) & (a < kflo + kfn))
    assert np.array_equal(kto, np.concatenate([[0], np.cumsum(cover)]))
    seen = np.zeros(K, np.int64)
    n_idx = 0
    for ti in range(len(lt)):
        q = np.arange(p0[ti], p1[ti])
        assert kfi0[ti] == n_idx
        for k in range(kflo[ti], kflo[ti] + kfn[ti]):
            e = kfl_off[ti] + (k - kflo[ti])
            want = (q[(pk[q] == k) & free[k]] - p0[ti]) if free[k] else np.zeros(0, np.int64)
            assert np.array_equal(lki[lko[e]:lko[e + 1]], want)
            assert lks[e] == kto[k] + seen[k]
            seen[k] += 1
        n_idx += int(np.sum(free[pk[q]]))
        assert lko[kfl_off[ti] + kfn[ti]] == n_idx and kfi_n[ti] == n_idx - kfi0[ti]

    # --- Schur and direct tiles
    s_target = (min(sz["SCHUR_TILE_LMS"], schur_lms) if schur_lms > 0
                else max(8, min(96, math.ceil(M / N_SM))))
    fb = [np.unique(kf_pb[pk[lp[i]:lp[i + 1]]]) for i in range(M)]
    fb = [x[x >= 0] for x in fb]
    wlo = np.array([x.min() if len(x) else -1 for x in fb])
    whi = np.array([x.max() if len(x) else -1 for x in fb])
    wide = (whi >= 0) & (whi - wlo + 1 > sz["SPAN_MAX"])
    st = t("schur_tiles").reshape(-1, 10)
    dt = t("direct_tiles").reshape(-1, 10)
    tiles = np.concatenate([st, dt]) if len(dt) else st
    tiles = tiles[np.argsort(tiles[:, 0], kind="stable")]
    a0, a1 = tiles[:, 0], tiles[:, 1]
    assert a0[0] == 0 and a1[-1] == M and np.array_equal(a0[1:], a1[:-1]) and np.all(a1 > a0)
    for tl in tiles:
        x0, x1, q0, q1, b0, b1, k_lo, span, direct, poff = tl
        assert (q0, q1, b0, b1) == (lp[x0], lp[x1], lb[x0], lb[x1])
        if direct:
            assert np.all(wide[x0:x1]) and (k_lo, span, poff) == (0, K - 1, -1)
            assert x1 - x0 <= sz["SCHUR_TILE_LMS"] and (x1 - x0 == 1 or lp[x1] - lp[x0] <= sz["SCHUR_TILE_PAIRS"])
            if x1 < M:
                assert (not wide[x1] or x1 - x0 >= sz["SCHUR_TILE_LMS"]
                        or lp[x1 + 1] - lp[x0] > sz["SCHUR_TILE_PAIRS"])
        else:
            assert not np.any(wide[x0:x1]) and x1 - x0 <= s_target
            assert np.all(wlo[x0:x1] == wlo[x0]) and np.all(whi[x0:x1] == whi[x0])
            if x1 < M:
                assert wide[x1] or wlo[x1] != wlo[x0] or whi[x1] != whi[x0] or x1 - x0 >= s_target
            has = whi[x0] >= 0
            assert (k_lo, span) == ((wlo[x0], whi[x0] - wlo[x0] + 1) if has else (0, 0))
    spans = st[:, 7].astype(np.int64)
    assert np.array_equal(st[:, 9], np.concatenate([[0], np.cumsum(spans * (spans + 1) * 18)[:-1]]))
    assert sz["max_span"] == max(1, int(spans.max(initial=0)))
    nfb = K - 1
    n_blk = nfb * (nfb + 1) // 2
    assert sz["n_blk"] == n_blk
    bto, bpa = t("blk_tiles_off"), t("blk_part_at")
    assert len(bto) == n_blk + 1 and bto[0] == 0
    for a in range(nfb):
        for b in range(a + 1):
            i = a * (a + 1) // 2 + b
            want = [tl[9] + 2 * ((a - tl[6]) * (a - tl[6] + 1) // 2 + (b - tl[6])) * 18
                    for tl in st if tl[6] <= b and a < tl[6] + tl[7]]
            assert bpa[bto[i]:bto[i + 1]].tolist() == want, (a, b)
    act = {i for i in range(n_blk) if bto[i + 1] > bto[i]} | {a * (a + 1) // 2 + a for a in range(nfb)}
    for tl in dt:
        for j in range(tl[0], tl[1]):
            x = fb[j]
            act |= {int(u * (u + 1) // 2 + v) for u in x for v in x if u >= v}
    assert t("act_blk").tolist() == sorted(act)

    # --- envelope of the factor
    n_c = 6 * (K - 1)
    npw = (n_c + 31) // 32 * 32
    assert (sz["n_c"], sz["npw"]) == (n_c, npw)
    assert sz["chol_blocked"] == int(chol_mode == 2 or (chol_mode == 0 and n_c >= 320))
    INF = 2 ** 31 - 1
    first_blk = np.full(nfb, INF)
    for x in fb:
        if len(x):
            first_blk[x] = np.minimum(first_blk[x], x.min())
    pe = t("panel_end", np.int16)
    for pn in range(sz["max_panels"]):
        if pn >= npw // 32:
            assert pe[pn] == 0
            continue
        rows = [i for i in range(32 * (pn + 1), n_c)
                if (i if first_blk[i // 6] == INF else 6 * first_blk[i // 6]) <= 32 * pn + 31]
        last = max(rows, default=32 * (pn + 1) - 1)
        assert pe[pn] == min(npw, (last + 1 + 31) // 32 * 32), pn

    # --- state in the device layouts, mirrors, zero buffers, control block
    rs, ps = sz["RIG_STRIDE"], sz["POSE_STRIDE"]

    def rig_layout(intr, T):
        out = np.zeros((C, rs))
        out[:, :4] = intr
        out[:, 4:13] = T[:, :, :3].reshape(C, 9)
        out[:, 13:16] = T[:, :, 3]
        return out.ravel()

    def pose_layout(T):
        return np.concatenate([T[:, :, :3].reshape(K, 9), T[:, :, 3]], axis=1).ravel()

    assert np.array_equal(t("rig", f64), rig_layout(w.intr, w.T_cb))
    assert np.array_equal(t("pose0", f64), pose_layout(w.poses))
    assert np.array_equal(t("lm0", f64), w.lms[lo].ravel())
    if prec == "mixed":
        assert np.array_equal(t("rig_f", np.float32), rig_layout(w.intr, w.T_cb).astype(np.float32))
        assert np.array_equal(t("pose_f0", np.float32), pose_layout(w.poses).astype(np.float32))
        assert np.array_equal(t("lm_f0", np.float32), w.lms[lo].ravel().astype(np.float32))
    for name in ("S", "dc", "dp", "lin_part", "bs_part"):
        assert np.all(t(name, f64) == 0), name
    assert t("ctrl", f64).tolist() == [0.0, 1e-4, 2.0]
    # --- replaced halves after the layout, and the read-back in the caller's layout
    assert np.array_equal(t("lm0_after_lms", f64), w.lms2[lo].ravel())
    assert np.array_equal(t("pose0_after_lms", f64), pose_layout(w.poses))
    assert np.array_equal(t("pose0_after_poses", f64), pose_layout(w.poses2))
    if prec == "mixed":
        assert np.array_equal(t("lm_f0_after_lms", np.float32), w.lms2[lo].ravel().astype(np.float32))
        assert np.array_equal(t("pose_f0_after_poses", np.float32), pose_layout(w.poses2).astype(np.float32))
    assert np.array_equal(t("got_lms", f64), w.lms2.ravel())
    assert np.array_equal(t("got_poses", f64), w.poses2.ravel())


@pytest.mark.parametrize("name,prec,lin_pairs,schur_lms,chol_mode", [
    ("c0", "fp64", 0, 0, 0),
    ("c1", "mixed", 0, 0, 0),
    ("c1", "fp64", 64, 16, 2),
    ("c2", "mixed", 0, 0, 0),
    ("wide", "mixed", 0, 0, 0),
    ("wide", "fp64", 32, 8, 1),
    ("two_keyframes", "fp64", 0, 0, 0),
    ("fixed_last", "mixed", 0, 0, 2),
    ("fixed_first_one_camera", "fp64", 32, 8, 0),
])
def test_host_tables_match_their_definitions(driver, tmp_path, name, prec, lin_pairs, schur_lms, chol_mode):
    small = {"two_keyframes": (2, 1, 3, 0), "fixed_last": (8, 3, 60, 7), "fixed_first_one_camera": (6, 1, 500, 0)}
    if name == "wide":
        w = wide_window()
    elif name in small:
        w = small_window(*small[name])
    else:
        w = Window.from_problem(synth.make_problem(name, 0))
    sz, t = run(driver, str(tmp_path), w, prec, lin_pairs, schur_lms, chol_mode)
    if name == "wide":
        assert len(t("direct_tiles")) > 0     # the window exercises direct tiles
    check_tables(w, sz, t, prec, lin_pairs, schur_lms, chol_mode)


def random_window(rng):
    """A random window: 2 to 40 keyframes, 1 to 4 cameras, 1 to 800 landmarks, most seen from a
    few nearby keyframes, some from keyframes spread over the window; every keyframe observed."""
    K, C, M = int(rng.integers(2, 41)), int(rng.integers(1, 5)), int(rng.integers(1, 801))
    kf, cam, lm = [], [], []
    for j in range(M):
        if rng.random() < 0.08:
            ks = rng.choice(K, size=int(rng.integers(min(2, K), K + 1)), replace=False)
        else:
            a = int(rng.integers(0, K))
            ks = np.clip(a + np.arange(int(rng.integers(1, 5))), 0, K - 1)
        views = [(int(k), int(rng.integers(0, C))) for k in ks for _ in range(int(rng.integers(1, 3)))]
        if len(views) < 2:
            views.append((int(ks[0]), int(rng.integers(0, C))))
        for k, c in views:
            kf.append(k), cam.append(c), lm.append(j)
    kf += list(range(K))                         # every keyframe observed, by landmark 0
    cam += [0] * K
    lm += [0] * K
    perm = rng.permutation(len(kf))
    kf, cam, lm = (np.asarray(a)[perm] for a in (kf, cam, lm))
    N = len(kf)
    intr = np.tile([350.0, 350.0, 200.0, 150.0], (C, 1))
    T_cb = np.tile(np.hstack([np.eye(3), np.zeros((3, 1))]), (C, 1, 1))
    poses = np.tile(np.hstack([np.eye(3), np.zeros((3, 1))]), (K, 1, 1))
    return Window(K, C, M, int(rng.integers(0, K)), kf, cam, lm, rng.normal(200, 30, (N, 2)), intr, T_cb, poses,
                  rng.normal(0, 4, (M, 3)), int(rng.integers(0, 1000)))


def test_host_tables_on_random_windows(driver, tmp_path):
    """24 seeded random windows, each with a random precision, tiling and factorisation mode."""
    rng = np.random.default_rng(77)
    for i in range(24):
        w = random_window(rng)
        prec = "mixed" if rng.random() < 0.5 else "fp64"
        lin = int(rng.choice([0, 32, 64, 128, 256]))
        schur = int(rng.choice([0, 8, 16, 32, 64, 128]))
        mode = int(rng.integers(0, 3))
        d = tmp_path / f"r{i}"
        d.mkdir()
        sz, t = run(driver, str(d), w, prec, lin, schur, mode)
        check_tables(w, sz, t, prec, lin, schur, mode)
