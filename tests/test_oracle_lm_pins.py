"""Pins for the oracle's LM control and its evaluation counts.

* Nielsen's damping update (H. B. Nielsen, IMM-REP-1999-05; also Madsen, Nielsen and
  Tingleff, "Methods for non-linear least squares problems", 2004, Sec. 3.2): literal
  values of the rule at chosen gains, a forced run of rejections, an accept after them.
* The accept rule: a step is taken iff the predicted reduction and the gain are positive,
  including gains below 0.25 that other LM variants would refuse.
* Inside the driver: near the optimum the residual is almost linear, so the quadratic model
  is almost exact, the gain is 1 to first order and the damping must fall by exactly 3.
* evaluate(): a hand-built window whose residuals are known exactly (0.5 px, exactly the
  Huber threshold, 2 px, one point behind the camera, one outside every index), so the
  cost, the RMS over valid observations only and the "e <= delta" inlier count are fixed by
  arithmetic done here by hand.
"""
import math

import numpy as np
import pytest

from oracle import ba
from paper_2506_04359_gb300 import synth


# ------------------------------------------------------------------ Nielsen's update

@pytest.mark.parametrize("gain, factor", [
    (1.0, 1.0 / 3.0),        # perfect model: 1 - 1 = 0, floored at 1/3
    (0.9, 1.0 / 3.0),        # 1 - 0.8^3 = 0.488 > 1/3 -> 0.488 (checked below exactly)
    (0.75, 0.875),           # 1 - 0.5^3
    (0.5, 1.0),              # 1 - 0^3: damping unchanged
    (0.25, 1.125),           # 1 - (-0.5)^3
    (0.1, 1.512),            # 1 - (-0.8)^3: a poor but accepted step raises lambda
    (1e-9, 2.0 - 6e-9),      # gain -> 0+: factor -> 2
])
def test_nielsen_accept_factors(gain, factor):
    if gain == 0.9:
        factor = 1.0 - 0.8 ** 3
    lam, nu = ba.nielsen_update(3.0, 16.0, gain, True)
    assert lam == pytest.approx(3.0 * factor, rel=1e-12)
    assert nu == 2.0                         # nu is reset after every accepted step


def test_nielsen_reject_sequence_doubles_nu():
    lam, nu = 1e-4, 2.0
    seen = []
    for _ in range(4):
        lam, nu = ba.nielsen_update(lam, nu, -0.5, False)
        seen.append((lam, nu))
    assert seen == [(2e-4, 4.0), (8e-4, 8.0), (6.4e-3, 16.0), (1.024e-1, 32.0)]
    lam, nu = ba.nielsen_update(lam, nu, 0.5, True)
    assert (lam, nu) == (1.024e-1, 2.0)


@pytest.mark.parametrize("L, F1, gain, ok", [
    (1.0, 0.0, 1e-3, True),      # tiny positive gain: accepted (no 0.25 threshold)
    (1.0, 0.0, 0.2, True),
    (1.0, 0.0, 0.0, False),      # no decrease
    (1.0, 0.0, -1.0, False),     # cost went up
    (0.0, 0.0, 1.0, False),      # no predicted reduction
    (-1.0, 0.0, 1.0, False),     # model predicts an increase
    (1.0, float("inf"), 1.0, False),
    (1.0, float("nan"), 1.0, False),
])
def test_accept_rule(L, F1, gain, ok):
    assert ba.accept_step(L, F1, gain) is ok


def test_driver_follows_the_rules_forced_rejections(monkeypatch):
    """Candidates made worse on purpose (every landmark moved 50 m) must all be rejected,
    lambda must go x2, x4, x8 and nu double, and the state must not move."""
    p = synth.make_problem("c0", M=60, K=3, seed=4)
    w = ba.Window.from_problem(p)
    real = ba.apply_step

    def worse(win, poses, lms, delta):
        P, L = real(win, poses, lms, delta)
        return P, L + 50.0

    monkeypatch.setattr(ba, "apply_step", worse)
    P, L, lam, nu, tr = ba.lm_solve(w, p.poses0, p.lm0, 4, lam0=1e-4)
    assert [r.accepted for r in tr] == [False] * 4
    assert [r.lam for r in tr] == [1e-4, 2e-4, 8e-4, 6.4e-3]
    assert (lam, nu) == (1.024e-1, 32.0)
    np.testing.assert_array_equal(P, p.poses0)
    np.testing.assert_array_equal(L, p.lm0)
    assert len({r.cost0 for r in tr}) == 1


def test_driver_gain_is_one_near_the_optimum():
    """A noise-free window a hair away from ground truth: the residual is linear to
    first order over the step, so the gain is 1 to ~1e-6 and lambda falls by exactly 3."""
    p = synth.make_problem("c0", M=80, K=4, seed=5, sigma=0.0)
    rng = np.random.default_rng(0)
    poses, lms = synth.perturb(p.poses_gt, p.lm_gt, rng, sigma_t=1e-7, sigma_r_deg=1e-6, sigma_l=1e-7)
    w = ba.Window.from_problem(p)
    lam0 = 1e-3
    _, _, lam, nu, tr = ba.lm_solve(w, poses, lms, 1, lam0=lam0)
    assert tr[0].accepted
    assert abs(tr[0].gain - 1.0) < 1e-4
    assert lam == lam0 / 3.0 and nu == 2.0


# --------------------------------------------------------------------------- evaluate

def _hand_window():
    """Two keyframes at the world origin (identity poses), one camera with fx = fy = 100 and
    cx = cy = 0 at the base: a landmark at (0, 0, 10) projects exactly to (0, 0)."""
    intr = np.array([[100.0, 100.0, 0.0, 0.0]])
    T_cb = np.zeros((1, 3, 4))
    T_cb[0, :, :3] = np.eye(3)
    lms = np.array([[0.0, 0.0, 10.0], [0.0, 0.0, 10.0], [0.0, 0.0, -3.0]])
    obs = [  # kf, lm, u, v  ->  r = pi(X) - o
        (0, 0, 0.5, 0.0),      # |r| = 0.5            inlier
        (1, 0, 1.0, 0.0),      # |r| = 1.0 = delta     inlier (e <= delta)
        (0, 1, 0.0, -2.0),     # |r| = 2.0            outlier
        (1, 1, 0.0, 0.0),      # |r| = 0              inlier
        (0, 2, 5.0, 5.0),      # behind the camera: invalid, no cost
        (1, 2, 5.0, 5.0),      # behind the camera: invalid, no cost
    ]
    o = np.array(obs, float)
    w = ba.Window(intr=intr, T_cb=T_cb, obs_kf=o[:, 0].astype(np.int64), obs_cam=np.zeros(len(obs), np.int64),
                  obs_lm=o[:, 1].astype(np.int64), obs_uv=o[:, 2:4].copy(), K=2, M=3, huber_delta=1.0)
    poses = np.zeros((2, 3, 4))
    poses[:, :, :3] = np.eye(3)
    return w, poses, lms


def test_evaluate_hand_window():
    w, poses, lms = _hand_window()
    ev = ba.evaluate(w, poses, lms)
    # rho: s for e <= 1, 2 e - 1 above: 0.25 + 1 + (4 - 1) + 0 = 4.25; F = 4.25 / 2
    assert ev.F == 2.125
    assert ev.n_valid == 4                 # the two points behind the camera do not count
    assert ev.n_inlier == 3                # e = 1.0 exactly is an inlier
    assert ev.rms == math.sqrt((0.25 + 1.0 + 4.0 + 0.0) / 4)    # over n_valid, not N


def test_evaluate_threshold_and_zmin_edges():
    w, poses, lms = _hand_window()
    # with delta just below 1 the e = 1 observation becomes an outlier: 2 * d * 1 - d^2
    d = 1.0 - 2.0 ** -20
    w.huber_delta = d
    ev = ba.evaluate(w, poses, lms)
    assert ev.n_inlier == 2
    assert ev.F == pytest.approx(0.5 * (0.25 + (2 * d - d * d) + (4 * d - d * d) + 0.0), rel=1e-15)
    # a point exactly at z_min is invalid (valid needs Z > z_min)
    w.huber_delta = 1.0
    w.z_min = 10.0
    assert ba.evaluate(w, poses, lms).n_valid == 0
    w.z_min = 10.0 - 1e-9
    assert ba.evaluate(w, poses, lms).n_valid == 4
