"""Batched windows (one launch per LM phase for all windows, one Cholesky cluster per
window, one graph per solve) against per-window solves and the oracle."""
import time

import numpy as np
import pytest

from oracle import ba
from paper_2506_04359_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cvba(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2506_04359_gb300 import cvba as m
    return m


@pytest.fixture(scope="module")
def windows():
    return synth.make_batch(12)


def test_batch_matches_single_window_solves_fp64(cvba, windows):
    iters = 6
    ctxs = [cvba.Context("fp64").load(p) for p in windows]
    batch = cvba.Batch(ctxs)
    for cs in (2, 8):
        batch.cvba_batch_set_chol_cluster(cs)
        for c, p in zip(ctxs, windows):
            c.cvba_set_poses(p.poses0, p.fixed_kf)
            c.cvba_set_landmarks(p.lm0)
        tr = batch.cvba_batch_solve(iters, huber_delta=1.0)
        for w, (c, p) in enumerate(zip(ctxs, windows)):
            single = cvba.Context("fp64").load(p)
            ts = single.cvba_solve(iters, huber_delta=1.0)
            assert tr[w]["accepted"].tolist() == ts["accepted"].tolist()
            assert np.all(np.abs(tr[w]["cost0"] - ts["cost0"]) <= 1e-10 * ts["cost0"])
            np.testing.assert_allclose(c.cvba_get_poses(), single.cvba_get_poses(), rtol=0, atol=1e-9)
            single.close()
    batch.close()


def test_batch_fp64_matches_oracle_on_sampled_windows(cvba, windows):
    iters = 10
    ctxs = [cvba.Context("fp64").load(p) for p in windows]
    batch = cvba.Batch(ctxs)
    tr = batch.cvba_batch_solve(iters)
    for w in (0, 5, 11):
        p = windows[w]
        P, L, _, _, otr = ba.lm_solve(ba.Window.from_problem(p), p.poses0, p.lm0, iters, keep_delta=False)
        assert tr[w]["accepted"].tolist() == [int(r.accepted) for r in otr]
        np.testing.assert_allclose(ctxs[w].cvba_get_poses(), P, rtol=0, atol=1e-6 * max(1.0, np.abs(P).max()))
        Lg = ctxs[w].cvba_get_landmarks()
        assert np.max(np.linalg.norm(Lg - L, axis=1) / np.linalg.norm(L, axis=1)) <= 1e-6
    batch.close()


def test_batch_mixed_rms_and_autotune(cvba, windows):
    iters = 10
    ctxs = [cvba.Context("mixed").load(p) for p in windows]
    batch = cvba.Batch(ctxs)
    cvba.lib.cvba_batch_autotune_clear()
    t0 = time.perf_counter()
    best = batch.cvba_batch_autotune(iters=2)
    t_tune = time.perf_counter() - t0
    assert best["lin_tile_pairs"] in (32, 64, 128, 256) and best["chol_cluster"] in (2, 4, 8, 16)
    assert best["schur_tile_landmarks"] in (8, 16, 32, 64, 128)
    t0 = time.perf_counter()
    again = batch.cvba_batch_autotune(iters=2)        # cached for this device and configuration
    assert again == best and time.perf_counter() - t0 < 0.5 * t_tune
    for c, p in zip(ctxs, windows):                     # autotune restored the initial state
        np.testing.assert_array_equal(c.cvba_get_poses(), p.poses0)
    batch.cvba_batch_solve(iters)
    for w in (1, 7):
        p = windows[w]
        win = ba.Window.from_problem(p)
        P, L, _, _, _ = ba.lm_solve(win, p.poses0, p.lm0, iters, keep_delta=False)
        rms_gpu = ba.evaluate(win, ctxs[w].cvba_get_poses(), ctxs[w].cvba_get_landmarks()).rms
        assert abs(rms_gpu - ba.evaluate(win, P, L).rms) <= 1e-3
    assert batch.cvba_batch_launch_count(iters) > 0
    batch.close()
