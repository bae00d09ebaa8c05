"""CPU checks of bench.py's own arithmetic: the per-result pose errors it reports against the
oracle, and the traffic record lookup that turns stale ncu counters into null."""
import hashlib
import json

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import bench


def _poses(rotvecs, trans):
    P = np.zeros((len(rotvecs), 3, 4))
    for i, (rv, t) in enumerate(zip(rotvecs, trans)):
        P[i, :, :3] = Rotation.from_rotvec(rv).as_matrix()
        P[i, :, 3] = t
    return P


@pytest.mark.parametrize("angle", [1e-9, 1e-4, 0.3, 3.1])
def test_pose_errors_recover_a_known_rotation_and_translation(angle):
    rng = np.random.default_rng(7)
    rv = rng.standard_normal((4, 3))
    t = rng.standard_normal((4, 3))
    Q = _poses(rv, t)
    axis = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    P = Q.copy()
    # keyframe 2: rotated by `angle` on the left, moved by 1e-3 m
    P[2, :, :3] = Rotation.from_rotvec(angle * axis).as_matrix() @ Q[2, :, :3]
    P[2, :, 3] += np.array([0.0, 6e-4, 8e-4])
    e = bench.pose_errors(P, Q)
    assert e["translation_m"] == pytest.approx(1e-3, rel=1e-9)
    assert e["rotation_rad"] == pytest.approx(angle, rel=1e-6, abs=1e-15)
    assert bench.pose_errors(Q, Q) == {"translation_m": 0.0, "rotation_rad": 0.0}


def test_traffic_record_is_null_once_the_kernel_source_changes(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel source, first version\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    rec = tmp_path / "traffic.json"
    rec.write_text(json.dumps({"k_x": {"workload": "w", "dram_bytes_per_launch": 123, "source_sha256": sha}}))
    monkeypatch.setattr(bench, "TRAFFIC", str(rec))
    monkeypatch.setattr(bench, "KERNEL_SOURCE", str(src))
    assert bench.traffic_of("k_x", "w") == 123
    assert bench.traffic_of("k_x", "another workload") is None
    assert bench.traffic_of("k_y", "w") is None
    src.write_text("kernel source, second version\n")
    assert bench.traffic_of("k_x", "w") is None
