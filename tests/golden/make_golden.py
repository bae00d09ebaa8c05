"""Write the oracle's results for the stored workloads (tests/golden/*.json).

Calls only oracle/ and the seeded input generator.  c0 and c1 come from the dense oracle
(oracle/ba.py); c4 (too large for a dense system) and the 256 windows of c3 from Oracle-S
(oracle/ba_sparse.py), whose pins tie it to the dense oracle.  Usage:
    python tests/golden/make_golden.py [c0 c1 c4 c3 ...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ba, ba_sparse  # noqa: E402
from paper_2506_04359_gb300 import synth  # noqa: E402


def _record(p, w, P, L, tr, dt, ev, ev0, source):
    return dict(workload=p.name, seed=p.seed, iters=p.iters, huber_delta=p.huber_delta, info=p.info,
                final_rms_px=ev.rms, final_cost=ev.F, final_n_valid=ev.n_valid, final_n_inlier=ev.n_inlier,
                initial_rms_px=ev0.rms,
                cost0=[r.cost0 for r in tr], accepted=[int(r.accepted) for r in tr],
                final_poses=P.tolist(), oracle_seconds=dt, source=source)


def golden(name: str) -> dict:
    p = synth.make_problem(name)
    w = ba.Window.from_problem(p)
    t = time.time()
    if name in ("c0", "c1"):
        P, L, lam, nu, tr = ba.lm_solve(w, p.poses0, p.lm0, p.iters, keep_delta=False)
        dt = time.time() - t
        return _record(p, w, P, L, tr, dt, ba.evaluate(w, P, L), ba.evaluate(w, p.poses0, p.lm0),
                       "oracle.ba.lm_solve (dense full normal equations, FP64)")
    sw = ba_sparse.SparseWindow(w)
    P, L, lam, nu, tr = ba_sparse.lm_solve(w, p.poses0, p.lm0, p.iters, keep_delta=False, sw=sw)
    dt = time.time() - t
    return _record(p, w, P, L, tr, dt, sw.evaluate(P, L), sw.evaluate(p.poses0, p.lm0),
                   "oracle.ba_sparse.lm_solve (block-sparse full normal equations, FP64)")


def golden_batch(n_windows: int = 256) -> dict:
    """Per-window results of the batched workload (windows of synth.make_batch)."""
    out = []
    t = time.time()
    for p in synth.make_batch(n_windows):
        w = ba.Window.from_problem(p)
        sw = ba_sparse.SparseWindow(w, threads=1)
        P, L, lam, nu, tr = ba_sparse.lm_solve(w, p.poses0, p.lm0, p.iters, keep_delta=False, sw=sw)
        ev = sw.evaluate(P, L)
        out.append(dict(seed=p.seed, K=p.K, M=p.M, N=p.N, final_rms_px=ev.rms, final_cost=ev.F,
                        cost0=[r.cost0 for r in tr], accepted=[int(r.accepted) for r in tr]))
        sw.close()
    return dict(workload="c3", n_windows=n_windows, iters=10, windows=out, oracle_seconds=time.time() - t,
                source="oracle.ba_sparse.lm_solve per window (block-sparse full normal equations, FP64)")


if __name__ == "__main__":
    for name in (sys.argv[1:] or ["c0", "c1", "c4", "c3"]):
        if name == "c3":
            g = golden_batch()
            with open(os.path.join(HERE, "c3_oracle.json"), "w") as f:
                json.dump(g, f, indent=1)
            print("c3", "oracle %.1f s" % g["oracle_seconds"])
            continue
        g = golden(name)
        with open(os.path.join(HERE, f"{name}_oracle.json"), "w") as f:
            json.dump(g, f, indent=1)
        print(name, "final rms %.9f px" % g["final_rms_px"], "oracle %.1f s" % g["oracle_seconds"])
