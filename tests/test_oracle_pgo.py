"""Pins for the pose-graph oracle, oracle/pgo.py.

* Log inverts Exp (oracle/ba.py's SE(3) exponential, itself pinned against the matrix
  exponential), across small angles and near pi.
* Edge Jacobians against central finite differences of the residual through left updates.
* A chain of odometry edges (a tree) has a zero-cost optimum, the dead-reckoned poses: LM
  started elsewhere reaches cost ~0 and those poses.
* Noise-free graphs with loops converge to the true poses from a perturbed start.
* Two poses, one edge, pose 0 fixed: the closed form T_1 = T_0 D.
"""
import numpy as np
import pytest

from oracle import ba, pgo
from paper_2506_04359_gb300 import synth


@pytest.mark.parametrize("mag", [0.0, 1e-9, 5e-5, 2e-4, 0.3, 2.0, 3.1, np.pi - 1e-7])
def test_log_inverts_exp(mag):
    rng = np.random.default_rng(int(mag * 1e3) % 1000)
    for _ in range(5):
        d = rng.normal(size=3)
        phi = mag * d / np.linalg.norm(d)
        xi = np.concatenate([rng.normal(size=3), phi])
        R, t = ba.se3_exp(xi)
        T = np.concatenate([R, t[:, None]], 1)
        np.testing.assert_allclose(pgo.se3_log(T), xi, atol=1e-9 if mag < 3.0 else 1e-6)


def test_edge_jacobians_match_central_differences():
    g = synth.make_pose_graph("pgo_loop", K=20)
    rng = np.random.default_rng(3)
    for e in (0, 5, g.E - 1):
        i, j = g.edges[e]
        Ti = ba.pose_plus(g.poses0[i], rng.normal(0, 0.05, 6))
        Tj = ba.pose_plus(g.poses0[j], rng.normal(0, 0.05, 6))
        r, Ji, Jj = pgo.edge_jacobians(Ti, Tj, g.deltas[e])
        h = 1e-6
        for which, J in ((0, Ji), (1, Jj)):
            fd = np.zeros((6, 6))
            for k in range(6):
                d = np.zeros(6)
                d[k] = h
                if which == 0:
                    rp = pgo.edge_residual(ba.pose_plus(Ti, d), Tj, g.deltas[e])
                    rm = pgo.edge_residual(ba.pose_plus(Ti, -d), Tj, g.deltas[e])
                else:
                    rp = pgo.edge_residual(Ti, ba.pose_plus(Tj, d), g.deltas[e])
                    rm = pgo.edge_residual(Ti, ba.pose_plus(Tj, -d), g.deltas[e])
                fd[:, k] = (rp - rm) / (2 * h)
            np.testing.assert_allclose(J, fd, atol=1e-7, rtol=1e-6)


def test_odometry_tree_reaches_the_dead_reckoned_poses():
    g = synth.make_pose_graph("pgo_loop", K=30, loop_every=0)      # odometry edges only
    assert g.E == g.K - 1
    rng = np.random.default_rng(1)
    start = g.poses0.copy()
    for k in range(1, g.K):
        start[k] = ba.pose_plus(start[k], rng.normal(0, 0.02, 6))
    P, lam, nu, tr = pgo.lm_solve(start, g.edges, g.deltas, 25)
    assert pgo.cost(P, g.edges, g.deltas) < 1e-16
    np.testing.assert_allclose(P, g.poses0, atol=1e-8)


def test_noise_free_loops_converge_to_the_truth():
    g = synth.make_pose_graph("pgo_loop", K=60, odo=(0.0, 0.0), loop=(0.0, 0.0))
    rng = np.random.default_rng(2)
    start = g.poses_gt.copy()
    for k in range(1, g.K):
        start[k] = ba.pose_plus(start[k], rng.normal(0, 0.05, 6))
    P, lam, nu, tr = pgo.lm_solve(start, g.edges, g.deltas, 30)
    np.testing.assert_allclose(P, g.poses_gt, atol=1e-8)
    costs = [r.cost0 for r in tr]
    assert all(b <= a for a, b in zip(costs, costs[1:]))


def test_single_edge_closed_form():
    g = synth.make_pose_graph("pgo_loop", K=2, loop_every=0)
    start = g.poses0.copy()
    start[1] = ba.pose_plus(start[1], np.array([0.3, -0.2, 0.1, 0.2, -0.1, 0.3]))
    P, lam, nu, tr = pgo.lm_solve(start, g.edges, g.deltas, 20)
    np.testing.assert_allclose(P[1], pgo.compose(P[0], g.deltas[0]), atol=1e-10)
