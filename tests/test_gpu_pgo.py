"""Pose-graph optimisation on the GPU against its oracle (oracle/pgo.py), through the C ABI
(cvba_pgo_solve): the two-lap loop (200 keyframes, 219 edges) and the four-lap map (600
keyframes), FP64.  The oracle's accept decisions (up to the first one below FP64
resolution, see parity_helpers) with per-iteration costs within 1e-9 relative; final poses
within 1e-6 (translation relative to max(|t|, 1 m), rotation in rad).  Edge cases: bad and
self edges, a free pose without edges, a short workspace."""
import numpy as np
import pytest

from oracle import pgo
from paper_2506_04359_gb300 import synth
from parity_helpers import compare_records

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cvba(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2506_04359_gb300 import cvba as m
    return m


def run_gpu(cvba, g, iters, edges=None, work_bytes=None):
    import torch
    dev = torch.device("cuda:0")
    t = lambda a, dt=torch.float64: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    ed = t(g.edges if edges is None else edges, torch.int32)
    de = t(g.deltas.reshape(g.E, 12))
    po = t(g.poses0.reshape(g.K, 12))
    need = cvba.cvba_pgo_workspace_bytes(g.K, g.E)
    work = torch.empty(need if work_bytes is None else work_bytes, dtype=torch.uint8, device=dev)
    trace = torch.zeros(max(iters, 1) * cvba.LM_RECORD_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    cvba.cvba_pgo_solve(g.K, g.E, ed.data_ptr(), de.data_ptr(), po.data_ptr(), iters, g.fixed, trace=trace.data_ptr(),
                        work=work.data_ptr(), work_bytes=work.numel(), stream=stream.cuda_stream)
    stream.synchronize()
    tr = np.frombuffer(trace.cpu().numpy().tobytes(), cvba.LM_RECORD_DTYPE)[:iters]
    return po.cpu().numpy().reshape(g.K, 3, 4), tr


def pose_err(P, Q):
    dt = np.linalg.norm(P[:, :, 3] - Q[:, :, 3], axis=1) / np.maximum(np.linalg.norm(Q[:, :, 3], axis=1), 1.0)
    E = np.einsum("kij,klj->kil", P[:, :, :3], Q[:, :, :3])
    s = np.linalg.norm(np.stack([E[:, 2, 1] - E[:, 1, 2], E[:, 0, 2] - E[:, 2, 0], E[:, 1, 0] - E[:, 0, 1]], 1), axis=1)
    return dt, np.arctan2(s / 2, (np.trace(E, axis1=1, axis2=2) - 1) / 2)


@pytest.mark.parametrize("name, iters", [("pgo_loop", 10), ("pgo_large", 5)])
def test_pgo_matches_oracle(cvba, name, iters):
    g = synth.make_pose_graph(name)
    P, tr = run_gpu(cvba, g, iters)
    Po, lam, nu, otr = pgo.lm_solve(g.poses0, g.edges, g.deltas, iters, fixed=g.fixed)
    n, worst = compare_records(tr, otr)
    dt, dr = pose_err(P, Po)
    print(f"{name}: {n} decisions compared, worst cost {worst:.2e}, translation {dt.max():.2e}, rotation "
          f"{dr.max():.2e}; cost {tr[0]['cost0']:.4e} -> {tr[-1]['cost0']:.4e}")
    assert dt.max() <= 1e-6 and dr.max() <= 1e-6
    assert np.array_equal(P[g.fixed], g.poses0[g.fixed])
    assert tr[-1]["cost0"] < 1e-2 * tr[0]["cost0"]


def test_pgo_edge_cases(cvba):
    g = synth.make_pose_graph("pgo_loop", K=20)
    for bad, status in (([[0, 25]], 2), ([[3, 3]], 2), ([[-1, 2]], 2)):
        ed = g.edges.copy()
        ed[4] = bad[0]
        with pytest.raises(cvba.CvbaError) as e:
            run_gpu(cvba, g, 3, edges=ed)
        assert e.value.status == status
    # pose 19 left without edges (the last odometry edge re-pointed to pose 17)
    ed = g.edges.copy()
    k = int(np.nonzero((ed[:, 1] == 19))[0][0])
    ed[k] = [17, 18] if ed[k, 0] != 17 else [16, 18]
    with pytest.raises(cvba.CvbaError) as e:
        run_gpu(cvba, g, 3, edges=ed)
    assert e.value.status == 1
    with pytest.raises(cvba.CvbaError) as e:
        run_gpu(cvba, g, 3, work_bytes=1024)
    assert e.value.status == 1
