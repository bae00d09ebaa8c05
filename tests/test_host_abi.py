"""The C ABI's host-side decisions on the CPU: tests/host_abi_driver.cpp calls the library
(cvba_host.cpp over a stand-in for the CUDA runtime; no kernel runs) in a fixed sequence on a
seeded window and records each status.  Checked: calls out of order (CVBA_ERR_STATE), invalid
sizes and options (CVBA_ERR_INVALID_ARG), indices out of range (CVBA_ERR_INDEX, naming the
first bad observation), non-finite values (CVBA_ERR_NONFINITE), a landmark left with one
observation, and the checkpoint: its size query, a round trip into a fresh context holding
another state of the same problem (poses, landmarks and damping restored), and the refusal
of a truncated buffer, a corrupted header and another problem's context; and when the captured
solve graph is reused or rebuilt."""
import os
import shutil
import subprocess
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from test_host_tables import Window  # noqa: E402

from paper_2506_04359_gb300 import synth  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2506_04359_gb300", "csrc")
OK, INVALID, INDEX, NONFINITE, CUDA, STATE = 0, 1, 2, 3, 4, 8

EXPECTED = {
    "create_bad_precision": INVALID, "create_bad_device": CUDA, "create": OK,
    "solve_before_setters": STATE, "observations_before_setters": STATE, "get_state_before_layout": STATE,
    "get_layout_before_layout": STATE,
    "rig_zero_cameras": INVALID, "rig_65_cameras": INVALID, "rig_nonfinite": NONFINITE,
    "rig_zero_image_size": INVALID, "rig": OK,
    "poses_one_keyframe": INVALID, "poses_257_keyframes": INVALID, "poses_fixed_out_of_range": INDEX,
    "poses_nonfinite": NONFINITE, "poses": OK,
    "landmarks_none": INVALID, "landmarks_nonfinite": NONFINITE, "landmarks_many": OK,
    "landmarks_many_nonfinite": NONFINITE, "landmarks": OK,
    "observations_camera_out_of_range": INDEX, "observations_landmark_negative": INDEX,
    "observations_keyframe_out_of_range": INDEX, "observations_nonfinite": NONFINITE,
    "observations_single_view_landmark": INVALID, "observations_none": INVALID, "observations": OK,
    "solve_negative_huber": INVALID, "solve_refine_9": INVALID, "solve_negative_iters": INVALID,
    "solve_nonfinite_zmin": INVALID, "chol_mode_3": INVALID, "tuning_negative": INVALID, "damping_set": OK,
    "chol_mode_2": OK, "solve_blocked": OK, "state_size": OK, "state_get": OK, "state_truncated": INVALID, "state_garbage": INVALID, "state_set": OK,
    "other_problem_layout": OK, "state_other_problem": INVALID,
}


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not cxx or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    out = str(tmp_path_factory.mktemp("adrv") / "host_abi_driver")
    base = [cxx, "-O1", "-g", "-std=c++17", "-pthread", "-I", cuda_inc, "-I", CSRC,
            os.path.join(ROOT, "tests", "host_abi_driver.cpp"), os.path.join(CSRC, "cvba_layout.cpp"), "-o", out]
    r = subprocess.run(base[:1] + ["-fsanitize=address"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base, check=True, capture_output=True)
    return out


def test_abi_statuses_and_checkpoint(driver, tmp_path):
    p = synth.make_problem("c0", 0)
    Window.from_problem(p).write(str(tmp_path))
    r = subprocess.run([driver, str(tmp_path)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    status, msg, extra = {}, {}, {}
    for line in open(tmp_path / "status.txt"):
        name, rest = line.rstrip("\n").split(" ", 1)
        if name in ("done", "state_bytes", "state_restored") or name.startswith("graphs_"):
            extra[name] = rest.split()
            continue
        code, _, text = rest.partition(" ")
        status[name], msg[name] = int(code), text
    assert extra["done"] == ["0"]
    assert status == EXPECTED
    # the first bad observation is named
    assert msg["observations_camera_out_of_range"].endswith("observation 3")
    assert msg["observations_landmark_negative"].endswith(f"observation {p.N - 1}")
    assert msg["observations_keyframe_out_of_range"].endswith("observation 0")
    assert "landmark 0" in msg["observations_single_view_landmark"]
    # checkpoint size query and full copy agree; poses, landmarks and damping restored
    n_query, n_got = (int(x) for x in extra["state_bytes"])
    assert n_query == n_got and n_query > 8 * (12 * p.K + 3 * p.M)
    flag, lam, nu = extra["state_restored"]
    assert flag == "1" and float(lam) == 0.5 and float(nu) == 3.0
    # the solve graph: reused for the same options and device view (new state values, the same
    # window loaded again into the same buffers, a tiling equal to the window's default sizes),
    # rebuilt for new options, another tiling or another factorisation
    graphs = {k: int(v[0]) for k, v in extra.items() if k.startswith("graphs_")}
    assert graphs == {"graphs_same": 1, "graphs_iters": 2, "graphs_new_state": 2, "graphs_same_window_again": 2,
                      "graphs_same_tuning": 2, "graphs_tuning": 3, "graphs_chol_mode": 4}
