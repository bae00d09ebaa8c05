"""Pins for Oracle-S, the block-sparse FP64 oracle (oracle/ba_sparse.py, oracle/ba_sparse.c).

Oracle-S solves the same damped normal equations as the dense oracle with a generic
block-sparse Cholesky, so it is pinned to the dense oracle (itself pinned in
test_oracle_pins.py / test_oracle_lm_pins.py) and to properties of sparse Cholesky:
* the normal equations it assembles: g and D equal the dense oracle's (1e-13);
* the increment: the dense oracle's solve at the same state (1e-12 relative while the
  system is far from the rounding floor of the residuals; the floor rule of the GPU parity
  tests afterwards), on c0, c1 and reduced versions of the multi-camera workloads;
* whole solves: c0 against the dense oracle; c1 against the stored dense-oracle results
  (tests/golden/c1_oracle.json): accept sequence, costs, final poses, RMS;
* the symbolic factorisation: every block the dense Cholesky factor of H has is in the
  pattern, and the pattern has no block the elimination-tree rule does not imply;
* a system that is not positive definite is reported, as the dense oracle reports it;
* results do not depend on the number of threads (bit for bit).
"""
import json
import os

import numpy as np
import pytest

from oracle import ba, ba_sparse
from paper_2506_04359_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def sparse_floor(sw, w, poses, lms, draws=4, seed=0):
    """Increment change from one-ulp rounding of the residuals, relative to |delta| (the
    floor used by the GPU parity tests), through Oracle-S's own factor."""
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
        acc += float(np.linalg.norm(sw.solve_rhs(dg[:-1]))) ** 2
    return np.sqrt(acc / draws)


def test_normal_equations_match_the_dense_oracle():
    p = synth.make_problem("c0", outlier_frac=0.1, seed=3)
    w = ba.Window.from_problem(p)
    sw = ba_sparse.SparseWindow(w)
    H, g, ev = ba.normal_equations(w, p.poses0, p.lm0)
    delta, D = ba.damped_solve(H, g, 1e-3)
    dS, DS, gS, evS = sw.linearise_solve(p.poses0, p.lm0, 1e-3)
    assert rel(gS, g) <= 1e-13 and rel(DS, D) <= 1e-13
    assert rel(dS, delta) <= 1e-12
    assert evS.n_valid == ev.n_valid and evS.n_inlier == ev.n_inlier
    assert abs(evS.F - ev.F) <= 1e-13 * ev.F and abs(evS.rms - ev.rms) <= 1e-13 * ev.rms
    # solve_rhs re-uses the factor: (H + lam D)^-1 b for another right-hand side
    b = np.random.default_rng(1).standard_normal(w.n_f)
    A = H + np.diag(1e-3 * D)
    assert rel(sw.solve_rhs(b), np.linalg.solve(A, b)) <= 1e-10


@pytest.mark.parametrize("name, kw", [
    ("c0", {}),
    ("c2", dict(K=10, M=2000)),
    ("c4", dict(K=10, M=2000)),
])
def test_lockstep_increment_matches_the_dense_oracle(name, kw):
    p = synth.make_problem(name, **kw)
    w = ba.Window.from_problem(p)
    sw = ba_sparse.SparseWindow(w)
    poses, lms, lam, nu, lin = p.poses0.copy(), p.lm0.copy(), 1e-4, 2.0, None
    n_it = 10 if name == "c0" else 3
    for it in range(n_it):
        dS, _, _, evS = sw.linearise_solve(poses, lms, lam)
        floor = sparse_floor(sw, w, poses, lms) / np.linalg.norm(dS)
        poses, lms, lam, nu, rec, lin = ba.lm_iteration(w, poses, lms, lam, nu, lin)
        d = rel(dS, rec.delta)
        assert d <= 1e-12 + 4.0 * floor, (name, it, d, floor)
        if it < 3:
            assert d <= 1e-11, (name, it, d)
        assert abs(evS.F - rec.cost0) <= 1e-13 * rec.cost0


def test_free_running_c0_matches_the_dense_oracle():
    p = synth.make_problem("c0")
    w = ba.Window.from_problem(p)
    P, L, lam, nu, tr = ba.lm_solve(w, p.poses0, p.lm0, p.iters)
    PS, LS, lamS, nuS, trS = ba_sparse.lm_solve(w, p.poses0, p.lm0, p.iters)
    assert [r.accepted for r in trS] == [r.accepted for r in tr]
    for a, b in zip(trS, tr):
        assert abs(a.cost0 - b.cost0) <= 1e-12 * b.cost0
        assert (a.n_valid, a.n_inlier) == (b.n_valid, b.n_inlier)
    assert np.abs(PS - P).max() <= 1e-10
    assert np.abs(LS - L).max() <= 1e-9 * np.abs(L).max()


def test_free_running_c1_matches_the_stored_dense_oracle():
    with open(os.path.join(HERE, "golden", "c1_oracle.json")) as f:
        gold = json.load(f)
    p = synth.make_problem("c1")
    w = ba.Window.from_problem(p)
    P, L, lam, nu, tr = ba_sparse.lm_solve(w, p.poses0, p.lm0, p.iters, keep_delta=False)
    assert [int(r.accepted) for r in tr] == gold["accepted"]
    c0 = np.array(gold["cost0"])
    assert np.abs(np.array([r.cost0 for r in tr]) - c0).max() <= 1e-12 * c0.min()
    assert np.abs(P - np.array(gold["final_poses"])).max() <= 1e-10
    ev = ba_sparse.SparseWindow(w).evaluate(P, L)
    assert abs(ev.rms - gold["final_rms_px"]) <= 1e-10
    assert (ev.n_valid, ev.n_inlier) == (gold["final_n_valid"], gold["final_n_inlier"])


def _block_order(w):
    """Dense column index of each block column of Oracle-S (landmarks first, then free
    keyframes) and its size."""
    cols = [np.arange(w.n_c + 3 * j, w.n_c + 3 * j + 3) for j in range(w.M)]
    cols += [np.arange(6 * b, 6 * b + 6) for b in range(w.K - 1)]
    return cols


@pytest.mark.parametrize("seed", [0, 1])
def test_symbolic_pattern_is_the_structural_fill(seed):
    """Permute the dense H to Oracle-S's block order, factor it densely and compare the
    nonzero blocks of the factor with the symbolic pattern; then check the pattern against
    a brute-force structural elimination (the graph rule: eliminating column c connects all
    its remaining neighbours)."""
    p = synth.make_problem("c2", K=6, M=40, seed=seed, track=(2, 4))
    w = ba.Window.from_problem(p)
    sw = ba_sparse.SparseWindow(w)
    cp, rows = sw.pattern()
    nb = sw.n_blocks
    pattern = {(int(r), c) for c in range(nb) for r in rows[cp[c]:cp[c + 1]]}
    H, g, _ = ba.normal_equations(w, p.poses0, p.lm0)
    D = ba.marquardt_diag(H)
    cols = _block_order(w)
    perm = np.concatenate(cols)
    A = (H + np.diag(1e-4 * D))[np.ix_(perm, perm)]
    Lf = np.linalg.cholesky(A)
    starts = np.cumsum([0] + [len(c) for c in cols])
    numeric = set()
    for c in range(nb):
        for r in range(c + 1, nb):
            if np.any(Lf[starts[r]:starts[r + 1], starts[c]:starts[c + 1]] != 0.0):
                numeric.add((r, c))
    assert numeric <= pattern
    # brute-force structural elimination on the block graph of H
    adj = [set() for _ in range(nb)]
    for c in range(nb):
        for r in range(c + 1, nb):
            if np.any(A[starts[r]:starts[r + 1], starts[c]:starts[c + 1]] != 0.0):
                adj[c].add(r)
                adj[r].add(c)
    struct = set()
    for c in range(nb):
        later = sorted(x for x in adj[c] if x > c)
        struct |= {(r, c) for r in later}
        for a in later:
            adj[a] |= {b for b in later if b != a}
    assert struct == pattern
    assert sw.n_indep == w.M


def test_not_positive_definite_is_reported():
    p = synth.make_problem("c0", M=50, K=3, seed=2)
    w = ba.Window.from_problem(p)
    sw = ba_sparse.SparseWindow(w)
    H, g, _ = ba.normal_equations(w, p.poses0, p.lm0)
    assert ba.damped_solve(H, g, -10.0)[0] is None
    assert sw.linearise_solve(p.poses0, p.lm0, -10.0)[0] is None


def test_thread_count_does_not_change_results():
    p = synth.make_problem("c2", K=12, M=3000)
    w = ba.Window.from_problem(p)
    out = []
    for t in (1, 3, 8):
        sw = ba_sparse.SparseWindow(w, threads=t)
        d, D, g, ev = sw.linearise_solve(p.poses0, p.lm0, 1e-4)
        out.append((d, g, ev.F))
        sw.close()
    for d, g, F in out[1:]:
        assert np.array_equal(d, out[0][0]) and np.array_equal(g, out[0][1]) and F == out[0][2]
