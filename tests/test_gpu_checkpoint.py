"""Checkpoint / resume of a solve through the C ABI, and the boundary's input checks.

Resuming is exact: on the FP64 path a solve of N iterations and a solve of k iterations,
a checkpoint (cvba_get_state), a restore (cvba_set_state, into the same or a fresh context)
and a solve of N - k iterations give bit-identical iteration records and final states.
"""
import numpy as np
import pytest

from paper_2506_04359_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cvba(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2506_04359_gb300 import cvba as m
    return m


@pytest.mark.parametrize("name, k", [("c0", 4), ("c1", 7)])
def test_resume_from_checkpoint_is_bit_exact_fp64(cvba, name, k):
    p = synth.make_problem(name)
    n = p.iters
    ref = cvba.Context("fp64").load(p)
    t_ref = ref.cvba_solve(n, huber_delta=p.huber_delta)
    P_ref, L_ref = ref.cvba_get_poses(), ref.cvba_get_landmarks()
    damp_ref = ref.cvba_get_damping()
    ref.close()

    a = cvba.Context("fp64").load(p)
    t1 = a.cvba_solve(k, huber_delta=p.huber_delta)
    state = a.cvba_get_state()
    # restore into a fresh context holding the same problem
    b = cvba.Context("fp64").load(p)
    b.cvba_set_state(state)
    t2 = b.cvba_solve(n - k, huber_delta=p.huber_delta, reset_lambda=False)
    trace = np.concatenate([t1, t2])
    for f in ("cost0", "cost1", "lambda", "gain", "pred", "step_norm", "accepted", "n_valid", "n_inlier"):
        assert np.array_equal(trace[f], t_ref[f], equal_nan=True), f
    assert np.array_equal(b.cvba_get_poses(), P_ref)
    assert np.array_equal(b.cvba_get_landmarks(), L_ref)
    assert b.cvba_get_damping() == damp_ref
    # and into the same context after it moved on
    a.cvba_solve(3, huber_delta=p.huber_delta, reset_lambda=False)
    a.cvba_set_state(state)
    a.cvba_solve(n - k, huber_delta=p.huber_delta, reset_lambda=False)
    assert np.array_equal(a.cvba_get_poses(), P_ref)
    assert np.array_equal(a.cvba_get_landmarks(), L_ref)
    a.close()
    b.close()


def test_checkpoint_rejects_another_problem(cvba):
    p = synth.make_problem("c0")
    q = synth.make_problem("c0", M=300, seed=3)
    a = cvba.Context("fp64").load(p)
    state = a.cvba_get_state()
    b = cvba.Context("fp64").load(q)
    with pytest.raises(cvba.CvbaError) as e:
        b.cvba_set_state(state)
    assert e.value.status == 1
    with pytest.raises(cvba.CvbaError) as e:
        b.cvba_set_state(b"not a checkpoint of anything at all" * 4)
    assert e.value.status == 1
    empty = cvba.Context("fp64")
    with pytest.raises(cvba.CvbaError) as e:
        empty.cvba_get_state()
    assert e.value.status == 8
    for c in (a, b, empty):
        c.close()


def test_free_keyframe_without_observations_is_rejected(cvba):
    p = synth.make_problem("c0", K=3, M=40)
    poses = np.concatenate([p.poses0, p.poses0[-1:]])       # a fourth keyframe nobody sees
    ctx = cvba.Context("fp64")
    ctx.cvba_set_rig(p.rig.intr, p.rig.T_cb)
    ctx.cvba_set_poses(poses, 0)
    ctx.cvba_set_landmarks(p.lm0)
    with pytest.raises(cvba.CvbaError) as e:
        ctx.cvba_set_observations(p.obs_kf, p.obs_cam, p.obs_lm, p.obs_uv)
    assert e.value.status == 1 and "keyframe 3" in str(e.value)
    # the same keyframe held fixed is fine: it has no columns
    ctx.cvba_set_poses(poses, 3)
    ctx.cvba_set_observations(p.obs_kf, p.obs_cam, p.obs_lm, p.obs_uv)
    ctx.close()


def test_rig_image_sizes_round_trip_and_checks(cvba):
    p = synth.make_problem("c0", M=40, K=3)
    ctx = cvba.Context("fp64").load(p)
    intr, T_cb, wh = ctx.cvba_get_rig()
    assert np.array_equal(intr, p.rig.intr) and np.array_equal(T_cb, p.rig.T_cb)
    assert np.array_equal(wh, p.rig.wh)
    with pytest.raises(cvba.CvbaError) as e:
        ctx.cvba_set_rig(p.rig.intr, p.rig.T_cb, np.zeros_like(p.rig.wh))
    assert e.value.status == 1
    ctx.cvba_set_rig(p.rig.intr, p.rig.T_cb)                  # sizes not given: zeros
    assert np.array_equal(ctx.cvba_get_rig()[2], np.zeros_like(p.rig.wh))
    ctx.close()
