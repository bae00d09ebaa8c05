"""GPU parity against the CPU oracle, through the C ABI.

FP64 path (the method itself): per-iteration solved increment within 1e-9 relative of the
oracle's full-system solve when both start from the same state and damping (lock-step);
free-running solves give the same accept/reject sequence, per-iteration costs within 1e-9
relative, and final poses / landmarks within 1e-6 relative; integer outputs (layout,
n_valid, n_inlier) are identical.  Mixed path: final RMS reprojection error within
1e-3 px of the oracle's.
"""
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


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def pose_errors(P, Q):
    """max translation error relative to max(|t|, 1 m) and max rotation error (rad)."""
    dt = max(np.linalg.norm(P[i, :, 3] - Q[i, :, 3]) / max(np.linalg.norm(Q[i, :, 3]), 1.0) for i in range(len(P)))
    dr = 0.0
    for i in range(len(P)):
        E = P[i, :, :3] @ Q[i, :, :3].T
        c = np.clip((np.trace(E) - 1.0) / 2.0, -1.0, 1.0)
        dr = max(dr, float(np.arccos(c)) if c < 1 - 1e-15 else float(np.linalg.norm(E - E.T) / (2 * np.sqrt(2))))
    return dt, dr


def rounding_floor(w, poses, lms, lam, draws=6, seed=0):
    """Increment change caused by one-ulp rounding of the residuals, relative to |delta|.

    r = fx X/Z + cx - o subtracts numbers of a few hundred pixels to leave ~1 px, so any
    two correct FP64 evaluations differ by ~2^-52 (|o| + |r| + |c|) per residual.  Near
    convergence g = J^T W r is a sum of nearly cancelling terms and this floor, mapped
    through (H + lam D)^-1, exceeds 1e-9 |delta|.  Returned: RMS over random one-ulp
    perturbations of |(H + lam D)^-1 J^T W e| / |delta|."""
    H, g, _ = ba.normal_equations(w, poses, lms)
    delta, D = ba.damped_solve(H, g, lam)
    A = H + np.diag(lam * D)
    r, _ = ba.residuals(w, poses, lms)
    _, wt = ba.huber(np.einsum("ni,ni->n", r, r), w.huber_delta)
    Jp, Jl = ba.jacobians(w, poses, lms)
    scale = 2.0 ** -52 * (np.abs(w.obs_uv) + np.abs(r) + np.abs(w.intr[w.obs_cam][:, 2:4]))
    pc = w.pose_col()[w.obs_kf]
    cols_p = np.where(pc[:, None] >= 0, pc[:, None] + np.arange(6), w.n_f)
    cols_l = w.n_c + 3 * w.obs_lm[:, None] + np.arange(3)
    rng = np.random.default_rng(seed)
    acc = 0.0
    for _ in range(draws):
        e = scale * rng.standard_normal(scale.shape)
        dg = np.zeros(w.n_f + 1)
        np.add.at(dg, cols_p, wt[:, None] * np.einsum("nai,na->ni", Jp, e))
        np.add.at(dg, cols_l, wt[:, None] * np.einsum("nai,na->ni", Jl, e))
        acc += float(np.linalg.norm(np.linalg.solve(A, dg[:-1]))) ** 2
    return np.sqrt(acc / draws) / float(np.linalg.norm(delta))


def lockstep(cvba, p, iters, precision="fp64", lam0=1e-4, lin_tile_pairs=0):
    """Drive GPU and oracle from the same state each iteration; return per-iteration
    (relative increment difference, allowed difference, gpu record, oracle record).
    Allowed: 1e-9 relative plus four times the residual-rounding floor."""
    w = ba.Window.from_problem(p)
    ctx = cvba.Context(precision).load(p)
    if lin_tile_pairs:
        ctx.cvba_set_tuning(lin_tile_pairs, 0)
    poses, lms, lam, nu = p.poses0.copy(), p.lm0.copy(), lam0, 2.0
    out = []
    for _ in range(iters):
        ctx.cvba_set_poses(poses, p.fixed_kf)
        ctx.cvba_set_landmarks(lms)
        ctx.cvba_set_damping(lam, nu)
        tr = ctx.cvba_solve(1, huber_delta=p.huber_delta, reset_lambda=False)
        dx = ctx.cvba_get_increment()
        tol = 1e-9 + 4.0 * rounding_floor(w, poses, lms, lam)
        poses, lms, lam, nu, rec, _ = ba.lm_iteration(w, poses, lms, lam, nu)
        out.append((rel(dx, rec.delta) if rec.delta is not None else 0.0, tol, tr[0], rec))
    ctx.close()
    return out


# --------------------------------------------------------------------- layout

@pytest.mark.parametrize("name", ["c0", "c1"])
def test_layout_is_bit_exact(cvba, name):
    p = synth.make_problem(name)
    ctx = cvba.Context("fp64").load(p)
    lo, oo, off = ctx.cvba_get_layout()
    rlo, roo, roff = ba.device_layout(p.obs_kf, p.obs_cam, p.obs_lm, p.M)
    assert np.array_equal(lo, rlo) and np.array_equal(oo, roo) and np.array_equal(off, roff)
    ctx.close()


# ------------------------------------------------------------------ FP64 path

def test_fp64_lockstep_increment_c0(cvba):
    p = synth.make_problem("c0")
    res = lockstep(cvba, p, p.iters)
    assert all(d <= 1e-9 for d, _, _, _ in res[:4])          # far from the rounding floor
    for d, tol, g, o in res:
        assert d <= tol, (d, tol)
        assert g["accepted"] == int(o.accepted)
        assert g["n_valid"] == o.n_valid and g["n_inlier"] == o.n_inlier
        assert abs(g["cost0"] - o.cost0) <= 1e-9 * o.cost0
        assert abs(g["cost1"] - o.cost1) <= 1e-9 * o.cost0


def test_fp64_free_running_c0(cvba):
    p = synth.make_problem("c0")
    w = ba.Window.from_problem(p)
    ctx = cvba.Context("fp64").load(p)
    tr = ctx.cvba_solve(p.iters, huber_delta=p.huber_delta)
    P, L, _, _, otr = ba.lm_solve(w, p.poses0, p.lm0, p.iters)
    assert tr["accepted"].tolist() == [int(r.accepted) for r in otr]
    c0 = np.array([r.cost0 for r in otr])
    np.testing.assert_array_less(np.abs(tr["cost0"] - c0), 1e-9 * c0 + 1e-300)
    assert tr["n_valid"].tolist() == [r.n_valid for r in otr]
    assert tr["n_inlier"].tolist() == [r.n_inlier for r in otr]
    dt, dr = pose_errors(ctx.cvba_get_poses(), P)
    assert dt <= 1e-6 and dr <= 1e-6
    Lg = ctx.cvba_get_landmarks()
    assert np.max(np.linalg.norm(Lg - L, axis=1) / np.linalg.norm(L, axis=1)) <= 1e-6
    ev = ctx.cvba_evaluate(p.huber_delta)
    oe = ba.evaluate(w, P, L)
    assert abs(ev["rms"] - oe.rms) <= 1e-9 and ev["n_valid"] == oe.n_valid and ev["n_inlier"] == oe.n_inlier
    ctx.close()


@pytest.mark.parametrize("kw", [dict(fixed_kf=2), dict(outlier_frac=0.2, seed=5), dict(M=37, K=3, seed=9)])
def test_fp64_lockstep_variants(cvba, kw):
    fixed = kw.pop("fixed_kf", 0)
    p = synth.make_problem("c0", **kw)
    p.fixed_kf = fixed
    for d, tol, g, o in lockstep(cvba, p, 4):
        assert d <= tol, (d, tol)
        assert g["accepted"] == int(o.accepted)


def test_fp64_lockstep_multicamera(cvba):
    """8-camera rig, 12 keyframes: several Schur tiles, windows and a ragged last tile."""
    p = synth.make_problem("c2", K=12, M=1500, seed=11)
    for d, tol, g, o in lockstep(cvba, p, 3):
        assert d <= tol, (d, tol)
        assert g["accepted"] == int(o.accepted)


def test_fp64_lockstep_wide_landmarks(cvba):
    """40 keyframes, distant points seen by every camera that sees them: most landmark
    windows are wider than a Schur tile window (24 keyframes), exercising the direct
    (atomic) Schur path next to the grouped one, and a 234-row reduced system."""
    p = synth.make_problem("c0", K=40, M=300, seed=14,
                           volume=dict(kind="box", lo=(-5.0, -2.0, 15.0), hi=(25.0, 2.0, 30.0)))
    for d, tol, g, o in lockstep(cvba, p, 3):
        assert d <= tol, (d, tol)
        assert g["accepted"] == int(o.accepted)


def test_fp64_lockstep_tiles_beyond_the_staged_observations(cvba):
    """Every observation of the 5-keyframe stereo window repeated eight times (a valid
    window: the same objective with each term weighted eight-fold), so a (landmark,
    keyframe) pair holds 16 observations, and tiles of 256 pairs hold more than the 1024
    observations a linearisation or back-substitution tile stages in shared memory: those
    tiles read their observations in place.  Increments, costs and decisions as the
    oracle's."""
    base = synth.make_problem("c0", M=200, seed=5)
    p = base.copy()
    p.obs_kf = np.repeat(base.obs_kf, 8)
    p.obs_cam = np.repeat(base.obs_cam, 8)
    p.obs_lm = np.repeat(base.obs_lm, 8)
    p.obs_uv = np.repeat(base.obs_uv, 8, axis=0)
    p.outlier = np.repeat(base.outlier, 8)
    n_pairs = np.unique(p.obs_lm.astype(np.int64) * p.K + p.obs_kf).size
    assert 256 * p.N / n_pairs > 2 * 1024
    for d, tol, g, o in lockstep(cvba, p, 3, lin_tile_pairs=256):
        assert d <= tol, (d, tol)
        assert g["accepted"] == int(o.accepted)
        assert abs(g["cost0"] - o.cost0) <= 1e-9 * o.cost0


@pytest.fixture(scope="module")
def c1_oracle():
    p = synth.make_problem("c1")
    w = ba.Window.from_problem(p)
    P, L, _, _, otr = ba.lm_solve(w, p.poses0, p.lm0, p.iters, keep_delta=False)
    return p, w, P, L, otr


def test_fp64_free_running_c1(cvba, c1_oracle):
    """20 keyframes, 5000 landmarks, 5% outliers: the oracle factors the dense 15k system."""
    p, w, P, L, otr = c1_oracle
    ctx = cvba.Context("fp64").load(p)
    tr = ctx.cvba_solve(p.iters, huber_delta=p.huber_delta)
    assert tr["accepted"].tolist() == [int(r.accepted) for r in otr]
    c0 = np.array([r.cost0 for r in otr])
    assert np.all(np.abs(tr["cost0"] - c0) <= 1e-9 * c0)
    assert tr["n_valid"].tolist() == [r.n_valid for r in otr]
    assert tr["n_inlier"].tolist() == [r.n_inlier for r in otr]
    dt, dr = pose_errors(ctx.cvba_get_poses(), P)
    assert dt <= 1e-6 and dr <= 1e-6
    Lg = ctx.cvba_get_landmarks()
    assert np.max(np.linalg.norm(Lg - L, axis=1) / np.linalg.norm(L, axis=1)) <= 1e-6
    ctx.close()


# ----------------------------------------------------------------- mixed path

def test_mixed_c1_rms_matches_oracle(cvba, c1_oracle):
    """Mixed precision: final RMS within 1e-3 px of the FP64 oracle; pose and landmark
    errors stated against the oracle's final state."""
    p, w, P, L, otr = c1_oracle
    ctx = cvba.Context("mixed").load(p)
    ctx.cvba_solve(p.iters, huber_delta=p.huber_delta)
    Pg, Lg = ctx.cvba_get_poses(), ctx.cvba_get_landmarks()
    rms_gpu = ba.evaluate(w, Pg, Lg).rms
    rms_or = ba.evaluate(w, P, L).rms
    dt, dr = pose_errors(Pg, P)
    dl = np.max(np.linalg.norm(Lg - L, axis=1))
    print(f"mixed c1: rms {rms_gpu:.6f} vs oracle {rms_or:.6f} px; pose dt {dt:.2e} (rel), dr {dr:.2e} rad; "
          f"max landmark error {dl:.2e} m")
    assert abs(rms_gpu - rms_or) <= 1e-3, (rms_gpu, rms_or)
    assert dt < 1e-3 and dr < 1e-3
    ctx.close()


# -------------------------------------------------------------------- errors

def test_error_paths(cvba):
    p = synth.make_problem("c0", M=20, K=3)
    ctx = cvba.Context("fp64")
    with pytest.raises(cvba.CvbaError) as e:
        ctx.cvba_solve(1)
    assert e.value.status == 8                               # solve before setters
    ctx.cvba_set_rig(p.rig.intr, p.rig.T_cb)
    ctx.cvba_set_poses(p.poses0)
    ctx.cvba_set_landmarks(p.lm0)
    bad = p.obs_cam.copy()
    bad[3] = 7
    with pytest.raises(cvba.CvbaError) as e:
        ctx.cvba_set_observations(p.obs_kf, bad, p.obs_lm, p.obs_uv)
    assert e.value.status == 2
    uv = p.obs_uv.copy()
    uv[1, 0] = np.nan
    with pytest.raises(cvba.CvbaError) as e:
        ctx.cvba_set_observations(p.obs_kf, p.obs_cam, p.obs_lm, uv)
    assert e.value.status == 3
    one = np.nonzero(p.obs_lm == 0)[0][1:]                   # landmark 0 left with one observation
    keep = np.setdiff1d(np.arange(p.N), one)
    with pytest.raises(cvba.CvbaError) as e:
        ctx.cvba_set_observations(p.obs_kf[keep], p.obs_cam[keep], p.obs_lm[keep], p.obs_uv[keep])
    assert e.value.status == 1
    ctx.cvba_set_observations(p.obs_kf, p.obs_cam, p.obs_lm, p.obs_uv)
    with pytest.raises(cvba.CvbaError) as e:
        ctx.cvba_solve(2, huber_delta=-1.0)
    assert e.value.status == 1
    ctx.close()


def test_invalid_observations_are_counted_exactly(cvba):
    """Points pushed behind some cameras: n_valid / n_inlier equal the oracle's."""
    p = synth.make_problem("c0", M=80, seed=12)
    lm0 = p.lm0.copy()
    lm0[:5, 2] = -3.0                                        # behind every camera of keyframe 0
    w = ba.Window.from_problem(p)
    ctx = cvba.Context("fp64").load(p, landmarks=lm0)
    ev = ctx.cvba_evaluate(p.huber_delta)
    oe = ba.evaluate(w, p.poses0, lm0)
    assert ev["n_valid"] == oe.n_valid < p.N
    assert ev["n_inlier"] == oe.n_inlier
    assert abs(ev["cost"] - oe.F) <= 1e-9 * oe.F
    ctx.close()
