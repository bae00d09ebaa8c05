"""The allocation-free evaluation entry point, checked against cvba_evaluate and the oracle.

cvba_evaluate_noalloc serves callers that cannot allocate device memory while running
(its scratch is a fixed device array inside the library).  This file is collected last,
so a run that stops at the first failure has already run every other test; it passes
both alone in a fresh process and after the other tests.  The comparison uses the same
tolerances as the parity tests: costs within 1e-9 relative, integer counts identical.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2506_04359_gb300 import synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cvba(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2506_04359_gb300 import cvba as m
    return m


def _device_inputs(p, lms, dev, kf=None, cam=None, lm=None):
    import torch
    f64 = lambda a: torch.tensor(np.ascontiguousarray(a, np.float64), device=dev)
    i32 = lambda a: torch.tensor(np.ascontiguousarray(a, np.int32), device=dev)
    return dict(intr=f64(p.rig.intr), tcb=f64(p.rig.T_cb.reshape(-1, 12)), poses=f64(p.poses0.reshape(p.K, 12)),
                land=f64(lms), kf=i32(p.obs_kf if kf is None else kf), cam=i32(p.obs_cam if cam is None else cam),
                lm=i32(p.obs_lm if lm is None else lm), uv=f64(p.obs_uv))


def _noalloc(cvba, p, t, dev, z_min=1e-3):
    import torch
    stream = torch.cuda.current_stream(dev)
    out = torch.full((5,), float("nan"), dtype=torch.float64, device=dev)
    cvba.cvba_evaluate_noalloc(p.N, p.K, p.C, p.M, t["intr"].data_ptr(), t["tcb"].data_ptr(), t["poses"].data_ptr(),
                               t["land"].data_ptr(), t["kf"].data_ptr(), t["cam"].data_ptr(), t["lm"].data_ptr(),
                               t["uv"].data_ptr(), p.huber_delta, z_min, out.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return out.cpu().numpy().tolist()


def test_noalloc_matches_context_evaluation_twice(cvba, cuda_device):
    p = synth.make_problem("c0", outlier_frac=0.1, seed=21)
    # move some landmarks behind the first keyframe so n_valid < n_obs is exercised
    lms = p.lm0.copy()
    lms[:7, 2] = -4.0
    ctx = cvba.Context("fp64").load(p, landmarks=lms)
    ref = ctx.cvba_evaluate(p.huber_delta)
    ctx.close()
    t = _device_inputs(p, lms, cuda_device)
    for call in range(2):
        cost, sq, nv, ni, bad = _noalloc(cvba, p, t, cuda_device)
        assert bad == 0.0, call
        assert int(nv) == ref["n_valid"] < p.N and int(ni) == ref["n_inlier"], call
        assert abs(cost - ref["cost"]) <= 1e-9 * ref["cost"], (call, cost, ref["cost"])
        assert abs(np.sqrt(sq / nv) - ref["rms"]) <= 1e-9 * ref["rms"], call


def test_noalloc_many_blocks_and_bad_indices_match_the_oracle(cvba, cuda_device):
    """284k observations (more than 256 partial blocks for the final reduction), with a few
    observations given out-of-range indices: those are counted and skipped, and the rest
    matches the oracle's evaluation of the valid observations."""
    from oracle import ba
    p = synth.make_problem("c2")
    kf, cam, lm = p.obs_kf.copy(), p.obs_cam.copy(), p.obs_lm.copy()
    bad = np.array([3, 1000, 77777, 150000, 284000])
    kf[bad[0]], cam[bad[1]], lm[bad[2]], kf[bad[3]], lm[bad[4]] = -1, p.C, p.M, p.K, -7
    keep = np.ones(p.N, bool)
    keep[bad] = False
    q = p.copy()
    q.obs_kf, q.obs_cam, q.obs_lm, q.obs_uv = p.obs_kf[keep], p.obs_cam[keep], p.obs_lm[keep], p.obs_uv[keep]
    ref = ba.evaluate(ba.Window.from_problem(q), p.poses0, p.lm0)
    t = _device_inputs(p, p.lm0, cuda_device, kf, cam, lm)
    for call in range(2):
        cost, sq, nv, ni, nbad = _noalloc(cvba, p, t, cuda_device)
        assert int(nbad) == bad.size, call
        assert int(nv) == ref.n_valid and int(ni) == ref.n_inlier, call
        assert abs(cost - ref.F) <= 1e-9 * ref.F, (call, cost, ref.F)
        assert abs(np.sqrt(sq / nv) - ref.rms) <= 1e-9 * ref.rms, call


def test_noalloc_rejects_oversize_and_bad_options(cvba, cuda_device):
    cases = [(4_194_305, 1.0, 1e-3, 1), (10, 1.0, 1e-3, 0), (10, float("inf"), 1e-3, 1),
             (10, -1.0, 1e-3, 1), (10, 1.0, float("-inf"), 1), (10, 1.0, float("nan"), 1)]
    for n, hub, zmin, ptr in cases:
        with pytest.raises(cvba.CvbaError) as e:
            cvba.cvba_evaluate_noalloc(n, 2, 1, 1, ptr, 1, 1, 1, 1, 1, 1, 1, hub, zmin, 1)
        assert e.value.status == 1, (n, hub, zmin, ptr)


@pytest.mark.parametrize("loading", ["EAGER", "LAZY"])
def test_noalloc_in_a_fresh_process(cvba, loading):
    """The first call in a fresh process, with the library's device module loaded eagerly
    (with the context) or lazily (by that first call)."""
    env = dict(os.environ, CUDA_MODULE_LOADING=loading)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.abspath(__file__), "-q", "-x", "-m", "gpu",
                        "-k", "matches_context_evaluation_twice", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "1 passed" in r.stdout
