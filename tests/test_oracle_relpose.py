"""Pins for the loop-closure relative-pose oracle, oracle/relpose.py.

* Left perturbations commute with the fixed map pose: Exp(xi) T^bm T^mw = Exp(xi) (T^bm T^mw),
  so every iterate of the relative-pose solve, composed with T^mw, is the motion-only solve's
  iterate from T^bw0 = T^bm0 T^mw (same accept decisions and costs until a decision falls
  below FP64 resolution, final poses to rounding).
* Noise-free queries: T^bm = T^bw_true (T^mw)^-1.
"""
import numpy as np

from oracle import pnp, relpose
from paper_2506_04359_gb300 import synth


def test_relative_pose_composed_with_the_map_pose_is_the_pnp_solve():
    b = synth.make_frames("pnp_multi", seed=2, frames=6)
    T_mw, T_bm0 = synth.make_map_poses(b, seed=1)
    rel = relpose.solve_queries(b, T_mw, T_bm0)
    abs_ = pnp.solve_frames(b)
    for f, ((Tbm, tr), (Tbw, tr2)) in enumerate(zip(rel, abs_)):
        # decisions are compared until the first one below FP64 resolution (|F - F'| <
        # 1e-12 F: the step changes nothing the cost can resolve, so both outcomes are right)
        for a, b_ in zip(tr, tr2):
            if abs(b_.cost0 - b_.cost1) < 1e-12 * b_.cost0:
                break
            assert a.accepted == b_.accepted
            assert abs(a.cost0 - b_.cost0) <= 1e-10 * b_.cost0
        np.testing.assert_allclose(relpose.compose(Tbm, T_mw[f]), Tbw, atol=1e-9)


def test_noise_free_query_recovers_the_relative_pose():
    b = synth.make_frames("pnp_stereo", seed=3, frames=4, sigma=0.0, outlier_frac=0.0)
    T_mw, T_bm0 = synth.make_map_poses(b, seed=2)
    for f, (Tbm, tr) in enumerate(relpose.solve_queries(b, T_mw, T_bm0, iters=15)):
        np.testing.assert_allclose(Tbm, relpose.compose(b.poses_gt[f], relpose.inverse(T_mw[f])), atol=1e-8)
        assert tr[-1].rms < 1e-6
