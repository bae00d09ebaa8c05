"""Pins for the motion-only bundle-adjustment (multi-camera PnP) oracle, oracle/pnp.py.

* Its normal equations are the pose block of the bundle-adjustment oracle's (already pinned
  against brute-force finite differences) for a window whose only free keyframe is the frame.
* Noise-free frames converge to the true pose.
* All-inlier optimum = scipy.optimize.least_squares (loss='linear') over the 6-vector twist.
* Huber optimum = scipy.optimize.least_squares on the per-observation residual norms with
  loss='huber', f_scale = delta, which is the same robust objective (scipy's cost
  1/2 C^2 rho(e^2 / C^2) equals 1/2 (e^2 for e <= C, 2 C e - C^2 above)).
* Accepted costs never increase.
"""
import numpy as np
import pytest
import scipy.optimize

from oracle import ba, pnp
from paper_2506_04359_gb300 import synth


def _frame(name="pnp_stereo", f=3, **kw):
    b = synth.make_frames(name, seed=1, frames=8, **kw)
    cam, lm, uv = b.frame(f)
    w = pnp.frame_window(b.rig.intr, b.rig.T_cb, b.lm, cam, lm, uv, b.huber_delta)
    return b, f, w


@pytest.mark.parametrize("name", ["pnp_stereo", "pnp_multi"])
def test_normal_equations_are_the_ba_pose_block(name):
    b, f, w = _frame(name)
    H, g, ev = pnp.normal_equations(w, b.poses0[f], b.lm)
    # the same observations in a two-keyframe window: keyframe 0 fixed (unobserved), keyframe 1 the frame
    w2 = ba.Window(intr=w.intr, T_cb=w.T_cb, obs_kf=np.ones(w.obs_cam.size, np.int64), obs_cam=w.obs_cam,
                   obs_lm=w.obs_lm, obs_uv=w.obs_uv, K=2, M=w.M, fixed_kf=0, huber_delta=w.huber_delta)
    used = np.unique(w.obs_lm)
    # keep the landmark set small for the dense system: renumber the used landmarks
    remap = -np.ones(w.M, np.int64)
    remap[used] = np.arange(used.size)
    w2.obs_lm = remap[w.obs_lm]
    w2.M = used.size
    poses = np.stack([b.poses0[f], b.poses0[f]])
    H2, g2, ev2 = ba.normal_equations(w2, poses, b.lm[used])
    np.testing.assert_allclose(H, H2[:6, :6], rtol=1e-12, atol=1e-12 * np.abs(H).max())
    np.testing.assert_allclose(g, g2[:6], rtol=1e-12, atol=1e-12 * np.abs(g).max())
    assert ev.F == pytest.approx(ev2.F, rel=1e-13) and ev.n_valid == ev2.n_valid


@pytest.mark.parametrize("name", ["pnp_stereo", "pnp_multi"])
def test_noise_free_frame_converges_to_the_true_pose(name):
    b, f, w = _frame(name, sigma=0.0, outlier_frac=0.0)
    T, lam, nu, tr = pnp.lm_solve(w, b.poses0[f], b.lm, 15)
    np.testing.assert_allclose(T, b.poses_gt[f], atol=1e-8)
    assert tr[-1].rms < 1e-6


def _twist_fun(w, T0, lms):
    def fun(x):
        r, _ = ba.residuals(w, ba.pose_plus(T0, x)[None], lms)
        return r.ravel()
    return fun


def test_inlier_optimum_matches_scipy_least_squares():
    b, f, w = _frame(outlier_frac=0.0)
    w.huber_delta = 1e6
    T, lam, nu, tr = pnp.lm_solve(w, b.poses0[f], b.lm, 30)
    sol = scipy.optimize.least_squares(_twist_fun(w, b.poses0[f], b.lm), np.zeros(6), loss="linear",
                                       xtol=1e-15, ftol=1e-15, gtol=1e-15)
    np.testing.assert_allclose(T, ba.pose_plus(b.poses0[f], sol.x), atol=1e-9)
    assert ba.evaluate(w, T[None], b.lm).F == pytest.approx(sol.cost, rel=1e-10)


@pytest.mark.parametrize("name", ["pnp_stereo", "pnp_multi"])
def test_huber_optimum_matches_scipy_huber_loss(name):
    b, f, w = _frame(name)
    T, lam, nu, tr = pnp.lm_solve(w, b.poses0[f], b.lm, 60)
    T0 = b.poses0[f]

    def norms(x):
        r, _ = ba.residuals(w, ba.pose_plus(T0, x)[None], b.lm)
        return np.sqrt(np.einsum("ni,ni->n", r, r))

    sol = scipy.optimize.least_squares(norms, np.zeros(6), loss="huber", f_scale=w.huber_delta, xtol=1e-15,
                                       ftol=1e-15, gtol=1e-15, max_nfev=2000)
    Ts = ba.pose_plus(T0, sol.x)
    F, Fs = ba.evaluate(w, T[None], b.lm).F, ba.evaluate(w, Ts[None], b.lm).F
    assert Fs == pytest.approx(sol.cost, rel=1e-12)
    assert F <= Fs * (1 + 1e-9)
    np.testing.assert_allclose(T, Ts, atol=1e-6)


def test_accepted_costs_do_not_increase_and_lambda_follows_the_rule():
    b, f, w = _frame("pnp_multi")
    T, lam, nu, tr = pnp.lm_solve(w, b.poses0[f], b.lm, 10)
    costs = [r.cost0 for r in tr]
    assert all(c1 <= c0 for c0, c1 in zip(costs, costs[1:]))
    l, n = 1e-4, 2.0
    for r in tr:
        assert r.lam == l
        l, n = ba.nielsen_update(l, n, r.gain, r.accepted)
