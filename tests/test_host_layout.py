"""The library's host layout (csrc/cvba_layout.cpp) on the CPU: compiled with the host
compiler into a small driver, run on seeded windows and compared exactly with the layout's
definition as the oracle states it (landmarks by (first, last observing keyframe, index);
observation slots by (landmark rank, keyframe, camera, index); segment offsets), with the
(landmark, keyframe) pairs derived here from that definition; plus the host worker pool under
nested and concurrent parallel sections."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import ba
from paper_2506_04359_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2506_04359_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not cxx or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    out = str(tmp_path_factory.mktemp("drv") / "host_layout_driver")
    subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-I", cuda_inc, "-I", CSRC,
                    os.path.join(ROOT, "tests", "host_layout_driver.cpp"), os.path.join(CSRC, "cvba_layout.cpp"),
                    "-o", out], check=True, capture_output=True)
    return out


def run_layout(driver, tmp, K, C, M, kf, cam, lm, fixed=0):
    N = len(kf)
    for stale in ("err.txt", "out.bin", "sizes.txt"):
        if os.path.exists(os.path.join(tmp, stale)):
            os.remove(os.path.join(tmp, stale))
    with open(os.path.join(tmp, "dims.txt"), "w") as f:
        f.write(f"{K} {C} {M} {N} {fixed}")
    for name, a in (("kf", kf), ("cam", cam), ("lm", lm)):
        np.asarray(a, np.int32).tofile(os.path.join(tmp, f"{name}.bin"))
    subprocess.run([driver, "layout", tmp], check=True)
    if os.path.exists(os.path.join(tmp, "err.txt")):
        return open(os.path.join(tmp, "err.txt")).read()
    P = int(open(os.path.join(tmp, "sizes.txt")).read())
    v = np.fromfile(os.path.join(tmp, "out.bin"), np.int32)
    sizes = [M, M, N, M + 1, N, P, P, P + 1, M + 1]
    parts = np.split(v, np.cumsum(sizes)[:-1])
    return dict(zip(["lm_order", "lm_rank", "obs_order", "lm_off", "obs_cam", "pair_kf", "pair_lm", "pair_obs",
                     "lm_pair"], parts))


def expected_pairs(kf, lm, lm_order, obs_order, M):
    """Pairs by the definition: the distinct (landmark rank, keyframe) runs of the slots."""
    rank = np.empty(M, np.int64)
    rank[lm_order] = np.arange(M)
    r = rank[np.asarray(lm)[obs_order]]
    k = np.asarray(kf)[obs_order]
    start = np.ones(len(obs_order), bool)
    start[1:] = (r[1:] != r[:-1]) | (k[1:] != k[:-1])
    s = np.nonzero(start)[0]
    lm_pair = np.searchsorted(r[s], np.arange(M + 1), side="left")
    return k[s], r[s], s, lm_pair


@pytest.mark.parametrize("name,seed", [("c0", 0), ("c1", 0), ("c0", 7)])
def test_host_layout_matches_the_definition(driver, tmp_path, name, seed):
    p = synth.make_problem(name, seed)
    # shuffle the caller's observation order further, so the sort has work at every level
    perm = np.random.default_rng(seed + 1).permutation(p.N)
    kf, cam, lm = p.obs_kf[perm], p.obs_cam[perm], p.obs_lm[perm]
    out = run_layout(driver, str(tmp_path), p.K, p.C, p.M, kf, cam, lm, p.fixed_kf)
    lo, oo, off = ba.device_layout(kf, cam, lm, p.M)
    assert np.array_equal(out["lm_order"], lo)
    assert np.array_equal(out["obs_order"], oo)
    assert np.array_equal(out["lm_off"], off)
    assert np.array_equal(out["lm_rank"][lo], np.arange(p.M))
    assert np.array_equal(out["obs_cam"], np.asarray(cam)[oo])
    pk, pl, po, lp = expected_pairs(kf, lm, lo, oo, p.M)
    assert np.array_equal(out["pair_kf"], pk) and np.array_equal(out["pair_lm"], pl)
    assert np.array_equal(out["pair_obs"][:-1], po) and out["pair_obs"][-1] == p.N
    assert np.array_equal(out["lm_pair"], lp)


@pytest.mark.parametrize("K,C,M,per_lm", [(256, 64, 3000, (2, 60)), (2, 1, 70000, (2, 3)), (40, 3, 1, (200, 201))])
def test_host_layout_matches_the_definition_at_the_limits(driver, tmp_path, K, C, M, per_lm):
    """The largest keyframe and camera counts the library accepts (both go into 8 bits of a
    sort key), many landmarks with two or three observations each (buckets of many
    landmarks), and a single landmark seen 200 times (one bucket, one group)."""
    rng = np.random.default_rng(K * 1000 + C)
    cnt = rng.integers(per_lm[0], per_lm[1], size=M)
    lm = np.repeat(np.arange(M), cnt)
    kf = rng.integers(0, K, size=len(lm))
    kf[:K] = np.arange(K) if len(lm) >= K else kf[:K]      # every keyframe observed
    cam = rng.integers(0, C, size=len(lm))
    perm = rng.permutation(len(lm))
    kf, cam, lm = kf[perm], cam[perm], lm[perm]
    out = run_layout(driver, str(tmp_path), K, C, M, kf, cam, lm, 0)
    assert not isinstance(out, str), out
    lo, oo, off = ba.device_layout(kf, cam, lm, M)
    assert np.array_equal(out["lm_order"], lo)
    assert np.array_equal(out["obs_order"], oo)
    assert np.array_equal(out["lm_off"], off)
    pk, pl, po, lp = expected_pairs(kf, lm, lo, oo, M)
    assert np.array_equal(out["pair_kf"], pk) and np.array_equal(out["pair_lm"], pl)
    assert np.array_equal(out["pair_obs"][:-1], po) and np.array_equal(out["lm_pair"], lp)


def test_host_layout_on_many_random_small_windows(driver, tmp_path):
    """120 seeded random windows (2 to 12 keyframes, 1 to 4 cameras, 1 to 300 landmarks with
    2 to 7 views each, now and then one with a single view, repeated (keyframe, camera) views,
    a random fixed keyframe, shuffled order): each layout equals the definition, and each
    refusal is one the definition calls for (a landmark with fewer than two observations, or a
    free keyframe with none)."""
    rng = np.random.default_rng(2024)
    n_rejected = 0
    for _ in range(120):
        K, C, M = int(rng.integers(2, 13)), int(rng.integers(1, 5)), int(rng.integers(1, 301))
        cnt = rng.integers(2, 8, size=M)
        if rng.random() < 0.15:                  # now and then a landmark seen once
            cnt[rng.integers(0, M)] = 1
        lm = np.repeat(np.arange(M), cnt)
        kf = rng.integers(0, K, size=len(lm))
        cam = rng.integers(0, C, size=len(lm))
        perm = rng.permutation(len(lm))
        kf, cam, lm = kf[perm], cam[perm], lm[perm]
        fixed = int(rng.integers(0, K))
        out = run_layout(driver, str(tmp_path), K, C, M, kf, cam, lm, fixed)
        counts = np.bincount(lm, minlength=M)
        seen = np.bincount(kf, minlength=K)
        should_reject = bool(np.any(counts < 2) or np.any((seen == 0) & (np.arange(K) != fixed)))
        if isinstance(out, str):
            assert should_reject, out
            n_rejected += 1
            continue
        assert not should_reject
        lo, oo, off = ba.device_layout(kf, cam, lm, M)
        assert np.array_equal(out["lm_order"], lo) and np.array_equal(out["obs_order"], oo)
        assert np.array_equal(out["lm_off"], off)
        pk, pl, po, lp = expected_pairs(kf, lm, lo, oo, M)
        assert np.array_equal(out["pair_kf"], pk) and np.array_equal(out["pair_lm"], pl)
        assert np.array_equal(out["pair_obs"][:-1], po) and np.array_equal(out["lm_pair"], lp)
    assert 0 < n_rejected < 120                  # both outcomes occur


def test_host_layout_rejections(driver, tmp_path):
    kf = [0, 1, 0, 1, 0]                     # landmark 2 has one observation
    cam = [0, 0, 1, 1, 0]
    lm = [0, 0, 1, 1, 2]
    assert "landmark 2" in run_layout(driver, str(tmp_path), 2, 2, 3, kf, cam, lm)
    kf = [0, 0, 0, 0]                        # keyframe 1 is free and unobserved
    assert "keyframe 1" in run_layout(driver, str(tmp_path), 2, 2, 2, kf, [0, 1, 0, 1], [0, 0, 1, 1])
    assert not isinstance(run_layout(driver, str(tmp_path), 2, 2, 2, kf, [0, 1, 0, 1], [0, 0, 1, 1], fixed=1), str)


def test_host_worker_pool_nested_and_concurrent(driver):
    r = subprocess.run([driver, "pool"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
