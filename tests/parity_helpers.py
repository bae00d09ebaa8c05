"""Shared comparison rules of the GPU parity tests.

Accept decisions follow the oracle's until the first decision the oracle takes below FP64
resolution (|F - F'| < 1e-12 F: the candidate changes nothing the cost can resolve, so
either outcome is correct and two correct FP64 programs may differ); the comparison stops
there (the LM reading's tie-break).
"""
import numpy as np


def compare_records(gpu, oracle, cost_rtol=1e-9):
    """gpu: structured records (cost0, accepted, n_valid, n_inlier fields); oracle: list of
    IterRecord.  Returns (iterations compared, worst relative cost0 difference); asserts on
    a mismatch."""
    worst = 0.0
    n = 0
    for g, o in zip(gpu, oracle):
        worst = max(worst, abs(float(g["cost0"]) - o.cost0) / max(abs(o.cost0), 1e-300))
        assert int(g["n_valid"]) == o.n_valid and int(g["n_inlier"]) == o.n_inlier, n
        if not (abs(o.cost0 - o.cost1) >= 1e-12 * abs(o.cost0)):
            break
        assert int(g["accepted"]) == int(o.accepted), n
        n += 1
    assert worst <= cost_rtol, worst
    return n, worst
