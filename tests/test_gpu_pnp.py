"""Motion-only bundle adjustment (multi-camera PnP) on the GPU against its oracle
(oracle/pnp.py), through the C ABI (cvba_pnp_solve).

FP64: every frame of both frame workloads (1024 stereo frames, 512 frames of the 32-camera
ring) takes the oracle's accept decisions (up to the first one below FP64 resolution, see
parity_helpers) with per-iteration costs within 1e-9 relative, integer counts identical, and
ends within 1e-6 of the oracle's pose (translation relative to max(|t|, 1 m), rotation in
rad).  FP32 inputs (the mixed path): every frame's final RMS within 1e-3 px of the oracle's,
poses within 1e-3 (relative) / 1e-4 rad.
Edge cases: empty frames, out-of-range indices, frames too large for shared-memory
staging, malformed segment offsets.
"""
import numpy as np
import pytest

from oracle import pnp
from paper_2506_04359_gb300 import synth
from parity_helpers import compare_records

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cvba(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2506_04359_gb300 import cvba as m
    return m


def run_gpu(cvba, b, dtype=0, iters=None, cam=None, lm=None, frame_off=None):
    import torch
    dev = torch.device("cuda:0")
    ft = torch.float64 if dtype == 0 else torch.float32
    t = lambda a, dt=ft: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    iters = b.iters if iters is None else iters
    intr, tcb, pw, uv = t(b.rig.intr), t(b.rig.T_cb.reshape(-1, 12)), t(b.lm), t(b.obs_uv)
    off = t(b.frame_off if frame_off is None else frame_off, torch.int32)
    cm = t(b.obs_cam if cam is None else cam, torch.int32)
    lmi = t(b.obs_lm if lm is None else lm, torch.int32)
    poses = t(b.poses0.reshape(b.F, 12), torch.float64)
    trace = torch.zeros(b.F * max(iters, 1) * cvba.LM_RECORD_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    cvba.cvba_pnp_solve(dtype, b.F, b.C, b.M, b.N, intr.data_ptr(), tcb.data_ptr(), pw.data_ptr(), off.data_ptr(),
                        cm.data_ptr(), lmi.data_ptr(), uv.data_ptr(), poses.data_ptr(), iters, b.huber_delta,
                        trace=trace.data_ptr(), stream=stream.cuda_stream)
    stream.synchronize()
    tr = np.frombuffer(trace.cpu().numpy().tobytes(), cvba.LM_RECORD_DTYPE).reshape(b.F, max(iters, 1))[:, :iters]
    return poses.cpu().numpy().reshape(b.F, 3, 4), tr


def pose_err(P, Q):
    """Translation error relative to max(|t|, 1 m) and rotation angle (rad), per frame."""
    dt = np.linalg.norm(P[:, :, 3] - Q[:, :, 3], axis=1) / np.maximum(np.linalg.norm(Q[:, :, 3], axis=1), 1.0)
    E = np.einsum("fij,fkj->fik", P[:, :, :3], Q[:, :, :3])
    s = np.linalg.norm(np.stack([E[:, 2, 1] - E[:, 1, 2], E[:, 0, 2] - E[:, 2, 0], E[:, 1, 0] - E[:, 0, 1]], 1), axis=1)
    dr = np.arctan2(s / 2, (np.trace(E, axis1=1, axis2=2) - 1) / 2)
    return dt, dr


@pytest.fixture(scope="module", params=["pnp_stereo", "pnp_multi"])
def frames(request):
    b = synth.make_frames(request.param)
    return b, pnp.solve_frames(b)


def test_fp64_matches_oracle_every_frame(cvba, frames):
    b, ref = frames
    P, tr = run_gpu(cvba, b, 0)
    worst_cost = 0.0
    for f, (T, otr) in enumerate(ref):
        _, w = compare_records(tr[f], otr)
        worst_cost = max(worst_cost, w)
        assert np.all(tr[f]["n_bad_index"] == 0)
    Po = np.stack([T for T, _ in ref])
    dt, dr = pose_err(P, Po)
    print(f"{b.name}: worst cost {worst_cost:.2e}, translation {dt.max():.2e} (rel), rotation {dr.max():.2e} rad; "
          f"frames beyond 1e-12: {int(np.sum((dt > 1e-12) | (dr > 1e-12)))}")
    assert worst_cost <= 1e-9
    assert dt.max() <= 1e-6 and dr.max() <= 1e-6


def test_fp32_inputs_match_oracle_pose_and_rms(cvba, frames):
    from oracle import ba
    b, ref = frames
    P, tr = run_gpu(cvba, b, 1)
    Po = np.stack([T for T, _ in ref])
    dt, dr = pose_err(P, Po)
    worst_rms = 0.0
    for f in range(b.F):
        cam, lm, uv = b.frame(f)
        w = pnp.frame_window(b.rig.intr, b.rig.T_cb, b.lm, cam, lm, uv, b.huber_delta)
        worst_rms = max(worst_rms, abs(ba.evaluate(w, P[f][None], b.lm).rms - ba.evaluate(w, Po[f][None], b.lm).rms))
    print(f"{b.name} fp32: translation {dt.max():.2e} (rel), rotation {dr.max():.2e} rad, rms {worst_rms:.2e} px")
    assert worst_rms <= 1e-3 and dt.max() <= 1e-3 and dr.max() <= 1e-4


def test_empty_frames_bad_indices_and_large_frames(cvba):
    from oracle import ba
    # frames 0..3 of a small batch; frame 1 emptied; frame 2 with bad indices
    b = synth.make_frames("pnp_stereo", seed=3, frames=4)
    keep = np.ones(b.N, bool)
    keep[b.frame_off[1]:b.frame_off[2]] = False
    q = synth.FrameBatch(**{**b.__dict__})
    q.obs_cam, q.obs_lm, q.obs_uv, q.outlier = b.obs_cam[keep], b.obs_lm[keep], b.obs_uv[keep], b.outlier[keep]
    cnt = np.diff(b.frame_off)
    cnt[1] = 0
    q.frame_off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
    cam, lm = q.obs_cam.copy(), q.obs_lm.copy()
    a2 = q.frame_off[2]
    bad = a2 + np.array([0, 5, 17])
    cam[bad[0]], lm[bad[1]], cam[bad[2]] = q.C, -1, -3
    P, tr = run_gpu(cvba, q, 0, cam=cam, lm=lm)
    assert np.all(tr[1]["nonpd"] == 1) and np.array_equal(P[1], q.poses0[1])
    assert np.all(tr[2]["n_bad_index"] == 3) and np.all(tr[0]["n_bad_index"] == 0)
    good = np.setdiff1d(np.arange(q.frame_off[2], q.frame_off[3]), bad)
    w = pnp.frame_window(q.rig.intr, q.rig.T_cb, q.lm, q.obs_cam[good], q.obs_lm[good], q.obs_uv[good], 1.0)
    T, _, _, otr = pnp.lm_solve(w, q.poses0[2], q.lm, q.iters)
    compare_records(tr[2], otr)
    assert np.abs(P[2] - T).max() <= 1e-6
    # frames beyond the shared-memory staging capacity (about 4,200 FP64 observations)
    big = synth.make_frames("pnp_multi", seed=4, frames=3, lm_per_frame=1500)
    assert np.diff(big.frame_off).min() > 5000
    P, tr = run_gpu(cvba, big, 0)
    for f, (T, otr) in enumerate(pnp.solve_frames(big)):
        compare_records(tr[f], otr)
        assert np.abs(P[f] - T).max() <= 1e-6


def test_malformed_offsets_are_rejected(cvba):
    b = synth.make_frames("pnp_stereo", seed=5, frames=4)
    for off in ([0, 10, 5, 20, b.N], [1, 10, 20, 30, b.N], [0, 10, 20, 30, b.N - 1]):
        with pytest.raises(cvba.CvbaError) as e:
            run_gpu(cvba, b, 0, frame_off=np.array(off, np.int32))
        assert e.value.status == 1


def test_relative_pose_matches_oracle_and_composes_to_the_pnp_pose(cvba):
    """Loop-closure queries (Sec. 2.3): map poses T^mw per frame; the solved T^bm against the
    relative-pose oracle, and T^bm T^mw against the motion-only solve of the same frames."""
    import torch
    from oracle import relpose
    b = synth.make_frames("pnp_multi", seed=6, frames=128)
    T_mw, T_bm0 = synth.make_map_poses(b, seed=3)
    dev = torch.device("cuda:0")
    t = lambda a, dt=torch.float64: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    intr, tcb, pw, uv = t(b.rig.intr), t(b.rig.T_cb.reshape(-1, 12)), t(b.lm), t(b.obs_uv)
    off, cm, lmi = t(b.frame_off, torch.int32), t(b.obs_cam, torch.int32), t(b.obs_lm, torch.int32)
    mw, bm = t(T_mw.reshape(b.F, 12)), t(T_bm0.reshape(b.F, 12))
    trace = torch.zeros(b.F * b.iters * cvba.LM_RECORD_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    cvba.cvba_relpose_solve(0, b.F, b.C, b.M, b.N, intr.data_ptr(), tcb.data_ptr(), pw.data_ptr(), off.data_ptr(),
                            cm.data_ptr(), lmi.data_ptr(), uv.data_ptr(), mw.data_ptr(), bm.data_ptr(), b.iters,
                            b.huber_delta, trace=trace.data_ptr(), stream=stream.cuda_stream)
    stream.synchronize()
    tr = np.frombuffer(trace.cpu().numpy().tobytes(), cvba.LM_RECORD_DTYPE).reshape(b.F, b.iters)
    Tbm = bm.cpu().numpy().reshape(b.F, 3, 4)
    ref = relpose.solve_queries(b, T_mw, T_bm0)
    for f, (T, otr) in enumerate(ref):
        compare_records(tr[f], otr)
    dt, dr = pose_err(Tbm, np.stack([T for T, _ in ref]))
    print(f"relative pose vs oracle: {dt.max():.2e} (rel), {dr.max():.2e} rad")
    assert dt.max() <= 1e-6 and dr.max() <= 1e-6
    Pw, _ = run_gpu(cvba, b, 0)
    comp = np.stack([relpose.compose(Tbm[f], T_mw[f]) for f in range(b.F)])
    dt, dr = pose_err(comp, Pw)
    print(f"relative pose composed with the map pose vs motion-only: {dt.max():.2e} (rel), {dr.max():.2e} rad")
    assert dt.max() <= 1e-6 and dr.max() <= 1e-6
    with pytest.raises(cvba.CvbaError) as e:
        cvba.cvba_relpose_solve(0, b.F, b.C, b.M, b.N, intr.data_ptr(), tcb.data_ptr(), pw.data_ptr(), off.data_ptr(),
                                cm.data_ptr(), lmi.data_ptr(), uv.data_ptr(), 0, bm.data_ptr(), b.iters)
    assert e.value.status == 1
