"""The allocation-free evaluation entry point, checked against cvba_evaluate.

cvba_evaluate_noalloc serves callers that cannot allocate device memory while running
(its scratch is a fixed device array inside the library).  This file is collected last,
so a run that stops at the first failure has already run every other test; it passes
both alone in a fresh process and after the other tests.  The comparison uses the same
tolerances as the parity tests: costs within 1e-9 relative, integer counts identical.
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


def test_noalloc_matches_context_evaluation_twice(cvba, cuda_device):
    import torch
    p = synth.make_problem("c0", outlier_frac=0.1, seed=21)
    # move some landmarks behind the first keyframe so n_valid < n_obs is exercised
    lms = p.lm0.copy()
    lms[:7, 2] = -4.0
    ctx = cvba.Context("fp64").load(p, landmarks=lms)
    ref = ctx.cvba_evaluate(p.huber_delta)
    ctx.close()

    dev = cuda_device
    f64 = lambda a: torch.tensor(np.ascontiguousarray(a, np.float64), device=dev)
    i32 = lambda a: torch.tensor(np.ascontiguousarray(a, np.int32), device=dev)
    intr, tcb = f64(p.rig.intr), f64(p.rig.T_cb.reshape(-1, 12))
    poses, land = f64(p.poses0.reshape(p.K, 12)), f64(lms)
    kf, cam, lm, uv = i32(p.obs_kf), i32(p.obs_cam), i32(p.obs_lm), f64(p.obs_uv)
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        out = torch.full((5,), float("nan"), dtype=torch.float64, device=dev)
        cvba.cvba_evaluate_noalloc(p.N, p.K, p.C, p.M, intr.data_ptr(), tcb.data_ptr(), poses.data_ptr(),
                                   land.data_ptr(), kf.data_ptr(), cam.data_ptr(), lm.data_ptr(), uv.data_ptr(),
                                   p.huber_delta, 1e-3, out.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        cost, sq, nv, ni, bad = out.cpu().numpy().tolist()
        assert bad == 0.0, call
        assert int(nv) == ref["n_valid"] < p.N and int(ni) == ref["n_inlier"], call
        assert abs(cost - ref["cost"]) <= 1e-9 * ref["cost"], (call, cost, ref["cost"])
        assert abs(np.sqrt(sq / nv) - ref["rms"]) <= 1e-9 * ref["rms"], call


def test_noalloc_rejects_oversize_and_null(cvba, cuda_device):
    with pytest.raises(cvba.CvbaError) as e:
        cvba.cvba_evaluate_noalloc(4_194_305, 2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1.0, 1e-3, 1)
    assert e.value.status == 1
    with pytest.raises(cvba.CvbaError) as e:
        cvba.cvba_evaluate_noalloc(10, 2, 1, 1, 0, 1, 1, 1, 1, 1, 1, 1, 1.0, 1e-3, 1)
    assert e.value.status == 1
