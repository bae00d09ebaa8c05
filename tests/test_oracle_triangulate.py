"""Pins for the multi-view triangulation oracle, oracle/triangulate.py.

* Noise-free observations: the linear (inhomogeneous DLT) point is the true landmark.
* Two noise-free views: the linear point equals the closed-form intersection of the two
  viewing rays (the midpoint of their common perpendicular, which has zero length).
* The refinement's normal equations are the landmark block of the bundle-adjustment oracle's
  (already pinned against brute-force finite differences).
* Refined optimum = scipy.optimize.least_squares over the 3 coordinates from the linear
  point: loss='linear' when every residual is an inlier; loss='huber' (f_scale = delta) on
  the per-observation norms, the same robust objective, when every fifth observation is
  moved 4-6 px (Huber outliers that leave the linear point in the right basin).
* Fewer than 2 observations and rank-deficient systems are reported, not raised.
"""
import numpy as np
import pytest
import scipy.optimize

from oracle import ba, triangulate as tri
from paper_2506_04359_gb300 import synth


def _segments(p):
    order, off = synth.landmark_segments(p.obs_lm, p.M)
    return order, off, p.obs_kf[order], p.obs_cam[order], p.obs_uv[order]


def _one(p, j, poses):
    order, off, kf, cam, uv = _segments(p)
    a, b = off[j], off[j + 1]
    return kf[a:b], cam[a:b], uv[a:b]


@pytest.mark.parametrize("name", ["c0", "c2"])
def test_noise_free_linear_point_is_the_landmark(name):
    p = synth.make_problem(name, sigma=0.0, outlier_frac=0.0, M=60, **({"K": 8} if name == "c2" else {}))
    order, off, kf, cam, uv = _segments(p)
    res = tri.triangulate(p.rig.intr, p.rig.T_cb, p.poses_gt, off, kf, cam, uv, iters=3)
    for j, (p0, pr, st, tr) in enumerate(res):
        assert st == tri.STATUS_OK
        np.testing.assert_allclose(p0, p.lm_gt[j], atol=1e-9 * max(1.0, np.abs(p.lm_gt[j]).max()))
        np.testing.assert_allclose(pr, p.lm_gt[j], atol=1e-9 * max(1.0, np.abs(p.lm_gt[j]).max()))


def test_two_views_intersect_like_the_rays():
    p = synth.make_problem("c0", sigma=0.0, M=30)
    for j in range(10):
        kf, cam, uv = _one(p, j, p.poses_gt)
        kf, cam, uv = kf[:2], cam[:2], uv[:2]
        R, t = tri.camera_from_world(p.rig.T_cb, p.poses_gt, kf, cam)
        c = -np.einsum("nji,nj->ni", R, t)                     # camera centres
        f = p.rig.intr[cam]
        d = np.einsum("nji,nj->ni", R, np.stack([(uv[:, 0] - f[:, 2]) / f[:, 0], (uv[:, 1] - f[:, 3]) / f[:, 1],
                                                  np.ones(2)], 1))
        # closest points c0 + s d0, c1 + u d1
        w0 = c[0] - c[1]
        A, B, C_ = d[0] @ d[0], d[0] @ d[1], d[1] @ d[1]
        D_, E = d[0] @ w0, d[1] @ w0
        den = A * C_ - B * B
        s, u = (B * E - C_ * D_) / den, (A * E - B * D_) / den
        mid = 0.5 * (c[0] + s * d[0] + c[1] + u * d[1])
        p0 = tri.linear(p.rig.intr, p.rig.T_cb, p.poses_gt, kf, cam, uv)
        np.testing.assert_allclose(p0, mid, rtol=0, atol=1e-8)


def test_normal_equations_are_the_ba_landmark_block():
    p = synth.make_problem("c2", K=8, M=40, seed=3)
    j = 7
    kf, cam, uv = _one(p, j, p.poses_gt)
    w = tri.landmark_window(p.rig.intr, p.rig.T_cb, kf, cam, uv, p.K, 1.0, 1e-3)
    pt = p.lm0[j] + 0.05
    r, valid = ba.residuals(w, p.poses_gt, pt[None])
    _, wt = ba.huber(np.einsum("ni,ni->n", r, r), 1.0)
    _, Jl = ba.jacobians(w, p.poses_gt, pt[None])
    H = np.einsum("n,nai,naj->ij", wt * valid, Jl, Jl)
    w2 = ba.Window(intr=w.intr, T_cb=w.T_cb, obs_kf=w.obs_kf, obs_cam=w.obs_cam, obs_lm=w.obs_lm, obs_uv=w.obs_uv,
                   K=p.K, M=1, fixed_kf=0, huber_delta=1.0)
    H2, g2, _ = ba.normal_equations(w2, p.poses_gt, pt[None])
    np.testing.assert_allclose(H, H2[w2.n_c:, w2.n_c:], rtol=1e-12, atol=1e-12 * np.abs(H).max())
    # and the refinement's first step solves that system
    p1, trc = tri.refine(w, p.poses_gt, pt, 1)
    g = np.einsum("n,nai,na->i", wt * valid, Jl, r)
    D = ba.marquardt_diag(H)
    np.testing.assert_allclose(trc[0].delta, np.linalg.solve(H + 1e-4 * np.diag(D), -g), rtol=1e-10)


def _norm_fun(w, poses):
    def fun(x):
        r, _ = ba.residuals(w, poses, x[None])
        return np.sqrt(np.einsum("ni,ni->n", r, r))
    return fun


@pytest.mark.parametrize("inliers", [True, False])
def test_refined_optimum_matches_scipy(inliers):
    p = synth.make_problem("c4", K=12, M=300, seed=2, outlier_frac=0.0)
    order, off, kf, cam, uv = _segments(p)
    hub = 1e6 if inliers else 1.0
    if not inliers:         # every fifth observation moved 4-6 px: Huber outliers the linear step survives
        uv = uv.copy()
        rng = np.random.default_rng(0)
        sel = np.arange(0, uv.shape[0], 5)
        ang = rng.uniform(0, 2 * np.pi, sel.size)
        uv[sel] += rng.uniform(4, 6, sel.size)[:, None] * np.stack([np.cos(ang), np.sin(ang)], 1)
    checked = 0
    for j in range(p.M):
        a, b = off[j], off[j + 1]
        if b - a < 4:
            continue
        w = tri.landmark_window(p.rig.intr, p.rig.T_cb, kf[a:b], cam[a:b], uv[a:b], p.K, hub, 1e-3)
        p0 = tri.linear(p.rig.intr, p.rig.T_cb, p.poses_gt, kf[a:b], cam[a:b], uv[a:b])
        pr, tr = tri.refine(w, p.poses_gt, p0, 40)
        if inliers:
            def fun(x):
                return ba.residuals(w, p.poses_gt, x[None])[0].ravel()
            sol = scipy.optimize.least_squares(fun, p0, loss="linear", xtol=1e-15, ftol=1e-15, gtol=1e-15)
        else:
            sol = scipy.optimize.least_squares(_norm_fun(w, p.poses_gt), p0, loss="huber", f_scale=hub, xtol=1e-15,
                                               ftol=1e-15, gtol=1e-15, max_nfev=2000)
        F, Fs = ba.evaluate(w, p.poses_gt, pr[None]).F, ba.evaluate(w, p.poses_gt, sol.x[None]).F
        if not inliers:
            # the robust objective is not convex: the LM point must be at least as good as
            # scipy's from the same start, and scipy started from the LM point must find
            # nothing lower than 1e-5 relative (IRLS converges linearly; a dropped or wrong
            # Huber weight moves the optimum's cost by percents)
            assert F <= Fs * (1 + 1e-9) + 1e-12
            sol = scipy.optimize.least_squares(_norm_fun(w, p.poses_gt), pr, loss="huber", f_scale=hub,
                                               xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=2000)
            Fs = ba.evaluate(w, p.poses_gt, sol.x[None]).F
        assert abs(F - Fs) <= (1e-9 if inliers else 1e-5) * Fs + 1e-12
        # positions agree to what the curvature resolves: |dp|_H^2 / 2 is a cost change
        r, valid = ba.residuals(w, p.poses_gt, pr[None])
        _, wt = ba.huber(np.einsum("ni,ni->n", r, r), hub)
        _, Jl = ba.jacobians(w, p.poses_gt, pr[None])
        H = np.einsum("n,nai,naj->ij", wt * valid, Jl, Jl)
        dp = pr - sol.x
        assert 0.5 * dp @ H @ dp <= (1e-8 if inliers else 1e-4) * Fs + 1e-12
        checked += 1
        if checked == 12:
            break
    assert checked == 12


def test_invalid_landmarks_are_reported():
    p = synth.make_problem("c0", M=20)
    order, off, kf, cam, uv = _segments(p)
    # landmark 0 with one observation; landmark 1 with two identical views (rank 2 at most)
    off2 = np.array([0, 1, 3], np.int32)
    kf2 = np.array([kf[0], kf[off[1]], kf[off[1]]])
    cam2 = np.array([cam[0], cam[off[1]], cam[off[1]]])
    uv2 = np.array([uv[0], uv[off[1]], uv[off[1]]])
    res = tri.triangulate(p.rig.intr, p.rig.T_cb, p.poses_gt, off2, kf2, cam2, uv2, iters=3)
    assert res[0][2] == tri.STATUS_FEW_OBS and np.all(np.isnan(res[0][1]))
    assert res[1][2] == tri.STATUS_DEGENERATE
