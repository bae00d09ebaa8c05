"""Pins for the oracle's differentiable cost: the SE(3) left Jacobian against finite
differences of the exponential's action on points, and every gradient against central
differences of the oracle's own cost (at a nonzero tangent perturbation)."""
import numpy as np
import pytest

from oracle import ba
from paper_2506_04359_gb300 import synth


def test_left_jacobian_matches_finite_differences_of_exp():
    rng = np.random.default_rng(0)
    for mag in [0.0, 5e-5, 0.3, 1.2]:
        xi = rng.normal(size=6)
        xi[3:] *= mag / max(np.linalg.norm(xi[3:]), 1e-300) if mag else 0.0
        X = rng.normal(size=3) * 3.0
        R, t = ba.se3_exp(xi)
        Xp = R @ X + t
        Jl = ba.se3_left_jacobian(xi)
        B = np.concatenate([np.eye(3), -ba.hat(Xp)], axis=1)       # d(Exp(d) X')/dd at d = 0
        h = 1e-6
        for k in range(6):
            e = np.zeros(6)
            e[k] = h
            Rp, tp = ba.se3_exp(xi + e)
            Rm, tm = ba.se3_exp(xi - e)
            fd = ((Rp @ X + tp) - (Rm @ X + tm)) / (2 * h)
            np.testing.assert_allclose(B @ Jl[:, k], fd, atol=1e-8 * max(1.0, np.abs(fd).max()))


def _problem():
    p = synth.make_problem("c2", K=4, M=15, track=(2, 4), seed=31, outlier_frac=0.2)
    rng = np.random.default_rng(5)
    xi = rng.normal(size=(p.K, 6)) * np.array([0.03, 0.03, 0.03, 0.02, 0.02, 0.02])
    return p, ba.Window.from_problem(p), xi


def test_cost_grad_matches_central_differences():
    p, w, xi = _problem()
    F, g = ba.cost_grad(w, p.poses0, p.lm0, p.rig.intr, xi)
    h = 1e-6

    def cost(poses=p.poses0, lms=p.lm0, intr=p.rig.intr, x=xi):
        return ba.cost_grad(w, poses, lms, intr, x)[0]

    def check(name, base, setter):
        fd = np.zeros_like(base)
        for idx in np.ndindex(base.shape):
            a, b = base.copy(), base.copy()
            a[idx] += h
            b[idx] -= h
            fd[idx] = (setter(a) - setter(b)) / (2 * h)
        np.testing.assert_allclose(g[name], fd, rtol=1e-5, atol=1e-5 * np.abs(fd).max(), err_msg=name)

    check("xi", xi, lambda v: cost(x=v))
    check("T", p.poses0, lambda v: cost(poses=v))
    check("lm", p.lm0, lambda v: cost(lms=v))
    check("intr", np.asarray(p.rig.intr, float), lambda v: cost(intr=v))


def test_cost_matches_evaluate_at_zero_perturbation():
    p, w, _ = _problem()
    F, g = ba.cost_grad(w, p.poses0, p.lm0)
    assert abs(F - ba.evaluate(w, p.poses0, p.lm0).F) <= 1e-12 * F
    # at xi = 0 the tangent gradient is the normal-equation gradient's pose block
    H, gg, _ = ba.normal_equations(ba.Window.from_problem(p), p.poses0, p.lm0)
    free = [i for i in range(p.K) if i != p.fixed_kf]
    np.testing.assert_allclose(g["xi"][free].ravel(), gg[:w.n_c], rtol=1e-10, atol=1e-10 * np.abs(gg).max())
    np.testing.assert_allclose(g["lm"].ravel(), gg[w.n_c:], rtol=1e-10, atol=1e-10 * np.abs(gg).max())
