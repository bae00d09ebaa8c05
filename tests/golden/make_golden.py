"""Write the oracle's results for the stored workloads (tests/golden/*.json).

Calls only oracle/ and the seeded input generator.  Usage:
    python tests/golden/make_golden.py [c0 c1 ...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ba  # noqa: E402
from paper_2506_04359_gb300 import synth  # noqa: E402


def golden(name: str) -> dict:
    p = synth.make_problem(name)
    w = ba.Window.from_problem(p)
    t = time.time()
    P, L, lam, nu, tr = ba.lm_solve(w, p.poses0, p.lm0, p.iters, keep_delta=False)
    dt = time.time() - t
    ev = ba.evaluate(w, P, L)
    return dict(workload=name, seed=p.seed, iters=p.iters, huber_delta=p.huber_delta, info=p.info,
                final_rms_px=ev.rms, final_cost=ev.F, final_n_valid=ev.n_valid, final_n_inlier=ev.n_inlier,
                initial_rms_px=ba.evaluate(w, p.poses0, p.lm0).rms,
                cost0=[r.cost0 for r in tr], accepted=[int(r.accepted) for r in tr],
                final_poses=P.tolist(), oracle_seconds=dt,
                source="oracle.ba.lm_solve (dense full normal equations, FP64)")


if __name__ == "__main__":
    for name in (sys.argv[1:] or ["c0", "c1"]):
        g = golden(name)
        with open(os.path.join(HERE, f"{name}_oracle.json"), "w") as f:
            json.dump(g, f, indent=1)
        print(name, "final rms %.9f px" % g["final_rms_px"], "oracle %.1f s" % g["oracle_seconds"])
