"""The batched solve's host logic on the CPU: cvba_host.cpp over a stand-in for the CUDA
runtime (host memory, no-op launchers, a counter of instantiated graphs, scripted event
timings), driven through the C ABI by tests/host_batch_driver.cpp on three windows of
different shapes (one with landmarks wider than a Schur tile's window).  Checked:

* a batch holding a window without a layout is refused (CVBA_ERR_STATE);
* the plan: every window's view as its context holds it, and the (window, item) work lists of
  each phase (linearisation tiles, keyframes, Schur tiles, active blocks, direct tiles,
  windows), in window order and item order, placed after the views on a 16-byte boundary;
* the captured graph is kept while nothing changes and rebuilt when the iteration count, a
  window's tiling or the Cholesky cluster size changes;
* the autotuner picks the fastest (linearisation tile, Schur tile) pair over its grid and then
  the fastest cluster size, leaves that tiling on every window, restores every window's state,
  answers a second call from its cache without timing, and times again after the cache is
  cleared."""
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from test_host_tables import Window, small_window, wide_window  # noqa: E402

from paper_2506_04359_gb300 import synth  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2506_04359_gb300", "csrc")
LIN = [32, 64, 128, 256]
SCHUR = [8, 16, 32, 64, 128]
CLUSTER = [2, 4, 8, 16]
CVBA_ERR_STATE = 8


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not cxx or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    out = str(tmp_path_factory.mktemp("bdrv") / "host_batch_driver")
    base = [cxx, "-O1", "-g", "-std=c++17", "-pthread", "-I", cuda_inc, "-I", CSRC,
            os.path.join(ROOT, "tests", "host_batch_driver.cpp"), os.path.join(CSRC, "cvba_layout.cpp"), "-o", out]
    r = subprocess.run(base[:1] + ["-fsanitize=address"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base, check=True, capture_output=True)
    return out


def script(best_pair, best_cs):
    """Elapsed times in the autotuner's order: the 20 (lin, schur) candidates, then the 4
    cluster sizes; the named ones fastest, ties broken by a slow ramp."""
    t = [2.0 + 0.01 * i for i in range(20)]
    t[LIN.index(best_pair[0]) * len(SCHUR) + SCHUR.index(best_pair[1])] = 1.0
    c = [3.0 + 0.01 * i for i in range(4)]
    c[CLUSTER.index(best_cs)] = 1.5
    return t + c


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_plan_graph_reuse_and_autotuner(driver, tmp_path, prec):
    wins = [Window.from_problem(synth.make_problem("c0", 0)), small_window(8, 3, 300, 7), wide_window()]
    for i, w in enumerate(wins):
        d = tmp_path / f"w{i}"
        d.mkdir()
        w.write(str(d))
    with open(tmp_path / "timings.txt", "w") as f:
        f.write(" ".join(str(x) for x in script((128, 64), 8) + script((64, 16), 2)))
    r = subprocess.run([driver, str(tmp_path), prec, str(len(wins))], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    out = {}
    for line in open(tmp_path / "out.txt"):
        k, *v = line.split()
        out[k] = [int(x) for x in v]
    assert out["done"] == [1]
    assert out["bare_status"] == [CVBA_ERR_STATE]
    # graph kept while nothing changes, rebuilt on each change
    assert out["graphs_after_first"] == [1] and out["graphs_after_same"] == [1]
    assert out["graphs_after_iters"] == [2] and out["graphs_after_tuning"] == [3]
    assert out["graphs_after_cluster"] == [4]
    assert out["chol_cs_first"] == [4] and out["chol_cs_tuned"] == [4] and out["chol_cs_cluster"] == [8]
    for tag in ("first", "tuned", "cluster"):
        assert out[f"views_equal_{tag}"] == [1] and out[f"lists_aligned_{tag}"] == [1]
        v = np.fromfile(tmp_path / f"lists_{tag}.bin", np.int32).reshape(-1, 3)
        tiles = [out[f"tiles_{tag}_{w}"] for w in range(len(wins))]
        counts = {0: 0, 1: 1, 2: 2, 3: 3, 4: 4}
        for phase, col in counts.items():
            got = v[v[:, 0] == phase][:, 1:]
            if phase == 3:                      # active blocks: per window its own ascending list
                assert np.array_equal(got[:, 0], np.repeat(np.arange(len(wins)), [t[3] for t in tiles]))
                for w, t in enumerate(tiles):
                    y = got[got[:, 0] == w][:, 1]
                    nfb = t[1] - 1
                    assert np.all(np.diff(y) > 0) and y.min() >= 0 and y.max() < nfb * (nfb + 1) // 2
                continue
            want = np.array([(w, i) for w, t in enumerate(tiles) for i in range(t[col])], np.int32).reshape(-1, 2)
            assert np.array_equal(got, want), (tag, phase)
        assert np.array_equal(v[v[:, 0] == 5][:, 1:], np.array([(w, 0) for w in range(len(wins))]))
    assert out["tiles_tuned_2"][0] > out["tiles_first_2"][0]      # 32-pair tiles on the last window
    assert sum(t[4] for t in (out[f"tiles_first_{w}"] for w in range(3))) > 0   # direct tiles in the plan
    # autotuner: pick, apply, restore; cached; timed again after a clear
    assert out["autotune_0"] == [128, 64, 8, 24, 1, 1, 8]
    assert out["autotune_1"] == [128, 64, 8, 0, 1, 1, 8]
    assert out["autotune_2"] == [64, 16, 2, 24, 1, 1, 2]
