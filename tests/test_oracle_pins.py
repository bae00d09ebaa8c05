"""Pins for the CPU oracle: each check ties it to something other than itself.

* SO(3)/SE(3) Exp: scipy's rotation-vector conversion and the matrix exponential of the
  4x4 twist (textbook special cases).
* Residual: zero at ground truth on noise-free synthetic data (the generator projects
  with its own camera-centre formula), principal point for a point on the optical axis.
* Jacobians: central finite differences of the residual through the SE(3) update.
* Normal equations: brute force J^T W J from a finite-difference Jacobian of the whole
  residual vector on a tiny window.
* Linear solve: numpy.linalg.solve.  Predicted reduction: the quadratic model evaluated
  directly.  Optimum: scipy.optimize.least_squares (loss='linear') when every residual
  is an inlier.  Gauge: a rigid change of world frame leaves costs and pose steps
  unchanged and rotates landmark steps.
* Planted mistakes (sign flip, dropped term, transposed rotation) in a copy of the oracle
  must fail these checks, so the checks have teeth.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.optimize
from scipy.spatial.transform import Rotation

from oracle import ba
from paper_2506_04359_gb300 import synth


def tiny(name="c0", seed=1, **kw):
    kw.setdefault("M", 8)
    if name == "c0":
        kw.setdefault("K", 3)
    return synth.make_problem(name, seed=seed, **kw)


def c2_tiny(seed=2, **kw):
    kw.setdefault("M", 12)
    kw.setdefault("K", 4)
    kw.setdefault("track", (2, 4))
    return synth.make_problem("c2", seed=seed, **kw)


# ------------------------------------------------------------------------ SE(3)

def test_so3_exp_matches_scipy():
    rng = np.random.default_rng(0)
    for mag in [0.0, 1e-9, 1e-6, 9.9e-5, 1.01e-4, 1e-3, 0.1, 1.0, 2.5, 3.1]:
        for _ in range(5):
            d = rng.normal(size=3)
            phi = mag * d / np.linalg.norm(d)
            R = ba.so3_exp(phi)
            np.testing.assert_allclose(R, Rotation.from_rotvec(phi).as_matrix(), atol=1e-13)
            np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-13)


def test_se3_exp_matches_matrix_exponential():
    rng = np.random.default_rng(1)
    for mag in [0.0, 5e-5, 2e-4, 0.3, 2.0]:
        for _ in range(4):
            rho = rng.normal(size=3)
            d = rng.normal(size=3)
            phi = mag * d / np.linalg.norm(d)
            A = np.zeros((4, 4))
            A[:3, :3] = ba.hat(phi) if mag else 0.0
            A[:3, 3] = rho
            E = scipy.linalg.expm(A)
            R, t = ba.se3_exp(np.concatenate([rho, phi]))
            np.testing.assert_allclose(R, E[:3, :3], atol=1e-12)
            np.testing.assert_allclose(t, E[:3, 3], atol=1e-12)


def test_exp_taylor_branch_is_continuous():
    d = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    lo, hi = ba.se3_exp(np.r_[1, 2, 3, (ba.TAYLOR_THETA * (1 - 1e-9)) * d]), \
        ba.se3_exp(np.r_[1, 2, 3, (ba.TAYLOR_THETA * (1 + 1e-9)) * d])
    np.testing.assert_allclose(lo[0], hi[0], atol=1e-15)
    np.testing.assert_allclose(lo[1], hi[1], atol=1e-15)


# --------------------------------------------------------------------- residual

@pytest.mark.parametrize("maker", [lambda: synth.make_problem("c0", sigma=0.0),
                                   lambda: c2_tiny(sigma=0.0, M=300)])
def test_zero_residual_at_ground_truth(maker):
    p = maker()
    w = ba.Window.from_problem(p)
    r, valid = ba.residuals(w, p.poses_gt, p.lm_gt)
    assert valid.all()
    assert np.abs(r).max() < 1e-9


def test_optical_axis_projects_to_principal_point():
    p = c2_tiny()
    poses = p.poses_gt
    kf, cam = 2, 5
    Rt = p.rig.T_cb[cam, :, :3] @ poses[kf, :, :3]                  # camera-from-world
    tt = p.rig.T_cb[cam, :, :3] @ poses[kf, :, 3] + p.rig.T_cb[cam, :, 3]
    centre = -Rt.T @ tt
    axis = Rt.T @ np.array([0.0, 0.0, 1.0])
    pt = centre + 7.0 * axis
    fx, fy, cx, cy = p.rig.intr[cam]
    w = ba.Window(intr=p.rig.intr, T_cb=p.rig.T_cb, obs_kf=np.array([kf]), obs_cam=np.array([cam]),
                  obs_lm=np.array([0]), obs_uv=np.array([[cx, cy]]), K=p.K, M=1)
    r, valid = ba.residuals(w, poses, pt[None])
    assert valid.all() and np.abs(r).max() < 1e-9


# ------------------------------------------------------------------- Jacobians

def jacobian_fd_error(mod, p, poses, lms, h=1e-6):
    """max |J - J_fd| / max(1, |J|) over all observations and columns."""
    w = ba.Window.from_problem(p)
    Jp, Jl = mod.jacobians(w, poses, lms)
    worst = 0.0
    for n in range(w.obs_kf.size):
        i, j = w.obs_kf[n], w.obs_lm[n]
        sub = ba.Window(intr=w.intr, T_cb=w.T_cb, obs_kf=w.obs_kf[n:n + 1], obs_cam=w.obs_cam[n:n + 1],
                        obs_lm=w.obs_lm[n:n + 1], obs_uv=w.obs_uv[n:n + 1], K=w.K, M=w.M)
        for c in range(6):
            e = np.zeros(6)
            e[c] = h
            Pp, Pm = poses.copy(), poses.copy()
            Pp[i] = ba.pose_plus(poses[i], e)
            Pm[i] = ba.pose_plus(poses[i], -e)
            fd = (ba.residuals(sub, Pp, lms)[0][0] - ba.residuals(sub, Pm, lms)[0][0]) / (2 * h)
            worst = max(worst, np.abs(fd - Jp[n, :, c]).max() / max(1.0, np.abs(Jp[n, :, c]).max()))
        for c in range(3):
            Lp, Lm = lms.copy(), lms.copy()
            Lp[j, c] += h
            Lm[j, c] -= h
            fd = (ba.residuals(sub, poses, Lp)[0][0] - ba.residuals(sub, poses, Lm)[0][0]) / (2 * h)
            worst = max(worst, np.abs(fd - Jl[n, :, c]).max() / max(1.0, np.abs(Jl[n, :, c]).max()))
    return worst


@pytest.mark.parametrize("maker", [tiny, c2_tiny])
def test_jacobians_match_central_differences(maker):
    p = maker()
    assert jacobian_fd_error(ba, p, p.poses0, p.lm0) < 1e-6


# ---------------------------------------------------------- normal equations

def full_fd_jacobian(w, poses, lms, h=1e-6):
    n_f = w.n_f
    r0, _ = ba.residuals(w, poses, lms)
    J = np.zeros((r0.size, n_f))
    for c in range(n_f):
        e = np.zeros(n_f)
        e[c] = h
        rp = ba.residuals(w, *ba.apply_step(w, poses, lms, e))[0].ravel()
        rm = ba.residuals(w, *ba.apply_step(w, poses, lms, -e))[0].ravel()
        J[:, c] = (rp - rm) / (2 * h)
    return J, r0


def normal_eq_brute_error(mod, p):
    w = ba.Window.from_problem(p)
    H, g, ev = mod.normal_equations(w, p.poses0, p.lm0)
    J, r = full_fd_jacobian(w, p.poses0, p.lm0)
    s = np.einsum("ni,ni->n", r, r)
    _, wt = ba.huber(s, w.huber_delta)
    W = np.repeat(wt, 2)
    Hb = J.T @ (W[:, None] * J)
    gb = J.T @ (W * r.ravel())
    return (np.abs(H - Hb).max() / np.abs(Hb).max(), np.abs(g - gb).max() / np.abs(gb).max())


@pytest.mark.parametrize("maker", [lambda: tiny(outlier_frac=0.25), lambda: c2_tiny(outlier_frac=0.2)])
def test_normal_equations_match_brute_force(maker):
    eh, eg = normal_eq_brute_error(ba, maker())
    assert eh < 1e-6 and eg < 1e-6


def test_fixed_keyframe_columns_are_absent():
    p = tiny()
    p.fixed_kf = 1
    w = ba.Window.from_problem(p)
    H, g, _ = ba.normal_equations(w, p.poses0, p.lm0)
    assert H.shape == (6 * 2 + 24, 6 * 2 + 24)
    J, r = full_fd_jacobian(w, p.poses0, p.lm0)
    _, wt = ba.huber(np.einsum("ni,ni->n", r, r), w.huber_delta)
    W = np.repeat(wt, 2)
    np.testing.assert_allclose(H, J.T @ (W[:, None] * J), rtol=1e-6, atol=1e-6 * np.abs(H).max())


def test_huber_weight_is_derivative_and_continuous():
    d = 1.3
    s = np.array([1e-4, 0.5, 1.0, d * d * (1 - 1e-6), d * d * (1 + 1e-6), 2.0, 9.0, 100.0])
    h = 1e-7
    rho, w = ba.huber(s, d)
    fd = (ba.huber(s + h, d)[0] - ba.huber(s - h, d)[0]) / (2 * h)
    np.testing.assert_allclose(w, fd, rtol=1e-5)
    # continuous at the threshold, quadratic below it
    assert abs(ba.huber(np.array([d * d]), d)[0][0] - d * d) < 1e-15
    np.testing.assert_allclose(rho[s < d * d], s[s < d * d])


def test_damped_solve_matches_numpy_and_model_decrease():
    p = tiny(outlier_frac=0.2)
    w = ba.Window.from_problem(p)
    H, g, ev = ba.normal_equations(w, p.poses0, p.lm0)
    lam = 3e-3
    delta, D = ba.damped_solve(H, g, lam)
    ref = np.linalg.solve(H + np.diag(lam * np.maximum(np.diag(H), 1e-12 * np.diag(H).max())), -g)
    np.testing.assert_allclose(delta, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())
    # predicted reduction equals the drop of the quadratic model F + g.d + 1/2 d.H.d
    L_formula = 0.5 * delta @ (lam * D * delta - g)
    L_model = -(g @ delta + 0.5 * delta @ H @ delta)
    assert abs(L_formula - L_model) <= 1e-9 * abs(L_model)


def test_marquardt_floor_applies_to_tiny_diagonals():
    H = np.diag([1e6, 1e-9, 0.0, 3.0])
    D = ba.marquardt_diag(H)
    np.testing.assert_allclose(D, [1e6, 1e-6, 1e-6, 3.0])


def test_nonpd_system_is_reported_not_raised():
    H = -np.eye(4)
    delta, _ = ba.damped_solve(H, np.ones(4), 1e-4)
    assert delta is None


# ------------------------------------------------------------------------- LM

def test_lm_costs_monotone_and_gradient_shrinks():
    p = synth.make_problem("c0")
    w = ba.Window.from_problem(p)
    P, L, lam, nu, tr = ba.lm_solve(w, p.poses0, p.lm0, 10)
    acc = [r.cost0 for r in tr] + [ba.evaluate(w, P, L).F]
    assert all(b <= a for a, b in zip(acc, acc[1:]))
    g0 = np.linalg.norm(ba.normal_equations(w, p.poses0, p.lm0)[1])
    g1 = np.linalg.norm(ba.normal_equations(w, P, L)[1])
    assert g1 < 1e-3 * g0


def test_noise_free_window_converges_to_ground_truth_cost():
    p = synth.make_problem("c0", sigma=0.0, seed=3)
    w = ba.Window.from_problem(p)
    P, L, lam, nu, tr = ba.lm_solve(w, p.poses0, p.lm0, 25)
    ev = ba.evaluate(w, P, L)
    assert ev.rms < 1e-6
    # gauge fixed at keyframe 0 -> the solution is the ground truth itself
    np.testing.assert_allclose(L, p.lm_gt, atol=1e-5)
    assert min(r.lam for r in tr) < tr[0].lam / 100     # lambda shrinks while converging


def _rigid(seed):
    r = np.random.default_rng(seed)
    Rs = Rotation.from_rotvec(r.normal(size=3) * 0.7).as_matrix()
    ts = r.normal(size=3) * 3.0
    return Rs, ts


@pytest.mark.parametrize("rotate,lam0", [(False, 1e-4), (True, 1e-13)])
def test_gauge_invariance_under_world_change(rotate, lam0):
    """A rigid change of world frame leaves costs and base-frame pose steps unchanged and
    rotates landmark steps.  Marquardt's diag(H) scaling is not rotation invariant in the
    landmark block, so the rotated case runs with negligible damping."""
    p = synth.make_problem("c0", M=60, seed=4, outlier_frac=0.1)
    w = ba.Window.from_problem(p)
    Rs, ts = _rigid(5)
    if not rotate:
        Rs = np.eye(3)
    poses2 = p.poses0.copy()
    poses2[:, :, :3] = p.poses0[:, :, :3] @ Rs.T
    poses2[:, :, 3] = p.poses0[:, :, 3] - np.einsum("kij,j->ki", poses2[:, :, :3], ts)
    lms2 = p.lm0 @ Rs.T + ts
    _, _, _, _, t1 = ba.lm_solve(w, p.poses0, p.lm0, 4, lam0=lam0)
    _, _, _, _, t2 = ba.lm_solve(w, poses2, lms2, 4, lam0=lam0)
    for a, b in zip(t1, t2):
        assert abs(a.cost0 - b.cost0) <= 1e-9 * a.cost0
        assert a.accepted == b.accepted
        tol = 1e-7 * np.abs(a.delta).max()
        np.testing.assert_allclose(b.delta[:w.n_c], a.delta[:w.n_c], rtol=0, atol=tol)
        dl1 = a.delta[w.n_c:].reshape(-1, 3) @ Rs.T
        np.testing.assert_allclose(b.delta[w.n_c:].reshape(-1, 3), dl1, atol=tol)


def test_inlier_optimum_matches_scipy_least_squares():
    p = tiny(M=10, K=3, seed=6)
    w = ba.Window.from_problem(p, huber_delta=1e6)      # every residual is an inlier
    P, L, lam, nu, tr = ba.lm_solve(w, p.poses0, p.lm0, 40)

    def fun(x):
        return ba.residuals(w, *ba.apply_step(w, p.poses0, p.lm0, x))[0].ravel()

    sol = scipy.optimize.least_squares(fun, np.zeros(w.n_f), loss="linear", xtol=1e-15, ftol=1e-15, gtol=1e-15)
    Fs = 0.5 * float(sol.fun @ sol.fun)
    Fo = ba.evaluate(w, P, L).F
    assert abs(Fo - Fs) <= 1e-8 * Fs
    Ps, Ls = ba.apply_step(w, p.poses0, p.lm0, sol.x)
    np.testing.assert_allclose(L, Ls, atol=1e-6)
    np.testing.assert_allclose(P, Ps, atol=1e-6)


# --------------------------------------------------------------------- layout

def test_layout_matches_python_sort():
    rng = np.random.default_rng(7)
    N, M = 500, 40
    kf = rng.integers(0, 6, N)
    cam = rng.integers(0, 3, N)
    lm = rng.integers(0, M, N)
    perm, off = ba.layout(kf, cam, lm, M)
    ref = sorted(range(N), key=lambda n: (lm[n], kf[n], cam[n], n))
    assert perm.tolist() == ref
    assert off.tolist() == [sum(1 for x in lm if x < j) for j in range(M + 1)]


# ------------------------------------------------------------ planted mistakes

class _Planted:
    """A copy of the oracle's Jacobian / normal-equation functions with one mistake."""

    def __init__(self, kind):
        self.kind = kind

    def jacobians(self, w, poses, lms):
        Jp, Jl = ba.jacobians(w, poses, lms)
        if self.kind == "sign_rot":
            Jp = Jp.copy()
            Jp[:, :, 3:] *= -1.0
        elif self.kind == "drop_rig":        # forgot R^cb in the chain
            Xb, Xc = ba.transform(w, poses, lms)
            Jp = Jp.copy()
            Jp[:, :, :3] = Jp[:, :, :3] @ np.linalg.inv(w.T_cb[w.obs_cam, :, :3])
        elif self.kind == "transpose_pose":  # R_i^T in place of R_i in dX_b/dp
            Rt = np.transpose(poses[w.obs_kf, :, :3], (0, 2, 1))
            Jl = Jl @ Rt @ Rt
        return Jp, Jl

    def normal_equations(self, w, poses, lms):
        H, g, ev = ba.normal_equations(w, poses, lms)
        if self.kind == "unweighted":        # dropped the Huber weight in g
            r, valid = ba.residuals(w, poses, lms)
            Jp, Jl = ba.jacobians(w, poses, lms)
            g = g.copy()
            pc = w.pose_col()[w.obs_kf]
            s = np.einsum("ni,ni->n", r, r)
            _, wt = ba.huber(s, w.huber_delta)
            for n in range(r.shape[0]):
                cl = w.n_c + 3 * w.obs_lm[n] + np.arange(3)
                g[cl] += (1.0 - wt[n]) * (Jl[n].T @ r[n])
        return H, g, ev


@pytest.mark.parametrize("kind", ["sign_rot", "drop_rig", "transpose_pose"])
def test_planted_jacobian_mistakes_are_caught(kind):
    p = c2_tiny()
    assert jacobian_fd_error(_Planted(kind), p, p.poses0, p.lm0) > 1e-3


def test_planted_weight_mistake_is_caught():
    eh, eg = normal_eq_brute_error(_Planted("unweighted"), tiny(outlier_frac=0.3, seed=8))
    assert eg > 1e-3


def test_normal_residual_matches_dense_system():
    """The matrix-free residual of the normal equations agrees with the dense H, g: ~0 for
    the dense Cholesky solution, the dense relative residual for a perturbed increment."""
    p = synth.make_problem("c0", 0)
    win = ba.Window.from_problem(p)
    H, g, _ = ba.normal_equations(win, p.poses0, p.lm0)
    lam = 1e-3
    delta, D = ba.damped_solve(H, g, lam)
    assert ba.normal_residual(win, p.poses0, p.lm0, lam, delta) <= 1e-12
    bad = delta.copy()
    bad[3] += 1e-3
    bad[win.n_c + 7] -= 2e-3
    A = H + np.diag(lam * D)
    dense = np.linalg.norm(A @ bad + g) / np.linalg.norm(g)
    assert dense > 1e-6
    assert abs(ba.normal_residual(win, p.poses0, p.lm0, lam, bad) - dense) <= 1e-9 * dense
