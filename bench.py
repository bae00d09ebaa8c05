"""Benchmark: LM iterations/s of sliding-window bundle adjustment on one GB300.

Default workload: the largest window (100 keyframes, a 32-camera ring of 16 stereo pairs,
200,000 landmarks, 3.75M observations with 3% outliers), mixed precision, 15 LM
iterations per solve; one step = one full solve from the same initial state.  The plain
FP64 path is timed on the same window beside it.

Prints one JSON line (rank 0).  Keys beyond the base contract: gobs_per_s; rms_px, the
oracle's RMS (stored Oracle-S result, tests/golden/<workload>_oracle.json) and the
validity gate |diff| <= 1e-3 px; vs_oracle (per-result error of the final state); fp64
(the FP64 path's throughput and error); roofline (dominant kernel) and roofline_all
(every kernel with a work model); cpu_baseline (Oracle-S on the host cores, a bounded
sample); e2e (through the public C API with host buffers); clocks; gpu_launches; and the
extra sections c1 (20-keyframe stereo window), batched (256 independent windows) and
small_solves (motion-only BA, loop-closure relative pose, triangulation, pose-graph
optimisation).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c4] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
KERNEL_SOURCE = os.path.join(ROOT, "paper_2506_04359_gb300", "csrc", "cvba_kernels.cu")
GOLDEN = os.path.join(ROOT, "tests", "golden")
METRIC = "BA LM iters/s & Gobs/s at RMS reproj within 1e-3 px of oracle; % HBM peak"
FALLBACK_HBM_GBS = 6800.0
FP64_NOMINAL_GFLOPS = 1250.0     # GB300 FP64 (non-tensor) nominal: 1.25 TFLOP/s
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12    # 80.5 TFLOP/s at the maximum SM clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c4")
    ap.add_argument("--precision", default=None, help="mixed (the workload's default) or fp64")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the c1 and batched c3 sections")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.rows = []
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 3 + k and r[3 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def pose_errors(P, Q) -> dict:
    """Largest keyframe translation error (m) and rotation error (rad, angle of R_P R_Q^T)."""
    dt = float(max(np.linalg.norm(P[i, :, 3] - Q[i, :, 3]) for i in range(len(P))))
    dr = 0.0
    for i in range(len(P)):
        E = P[i, :, :3] @ Q[i, :, :3].T
        s = np.linalg.norm(np.array([E[2, 1] - E[1, 2], E[0, 2] - E[2, 0], E[1, 0] - E[0, 1]])) / 2.0
        c = (np.trace(E) - 1.0) / 2.0
        dr = max(dr, float(np.arctan2(s, c)))
    return {"translation_m": dt, "rotation_rad": dr}


# -------------------------------------------------------------- algorithmic work model

def work_model(p, P: int, mixed: bool) -> dict:
    """Work of each kernel of one LM iteration: per-unit figures x units.

    "bytes" are the ALGORITHMIC bytes (what the method itself must move, with the
    linearisation, Schur and back-substitution fused and no per-pair intermediate in HBM):
    per observation its pixel (2 values) and a packed keyframe/camera index (4 B), read once
    by the linearisation and once by the candidate-cost pass; per landmark its position read
    by the linearisation (3 values + 4 B segment offset) and by the candidate pass, which also
    writes the candidate (FP64, plus its FP32 mirror on the mixed path).  "impl_bytes" add what
    this implementation moves besides: the 9-value summary of each (landmark, keyframe) pair
    and its index, written by the linearisation and read by the Schur and back-substitution
    kernels, and the landmark blocks (H_ll, g_l, V^-1).  The Schur complement and the reduced
    system's factorisation are arithmetic-bound: FP32 (mixed) or FP64 FLOPs, with
    m_j(m_j+1)/2 x 216 + m_j x 108 per landmark (m_j free keyframes observing it) and
    n_c^3/3 + 2 n_c^2."""
    t = 4 if mixed else 8
    N, M, K = p.N, p.M, p.K
    n_c = 6 * (K - 1)
    free = np.asarray(p.obs_kf) != p.fixed_kf
    keys = np.unique(p.obs_lm[free].astype(np.int64) * K + p.obs_kf[free])
    m = np.bincount(keys // K, minlength=M).astype(np.float64)
    blocks = float(np.sum(m * (m + 1) / 2))
    obs = N * (2 * t + 4)
    lm_lin = M * (3 * t + 4)
    lm_back = M * (3 * t + 4 + 24 + (12 if mixed else 0))
    pair = P * (4 + 9 * t)
    return {
        "lin": {"bytes": obs + lm_lin, "impl_bytes": obs + lm_lin + pair + M * 9 * t + K * 96,
                "flops": 110.0 * N + 130.0 * P},
        "schur_group": {"bytes": 8 * n_c * n_c, "impl_bytes": pair + M * 15 * t + 8 * n_c * n_c,
                        "flops": 216.0 * blocks + 108.0 * float(np.sum(m)), "fp32": mixed},
        "chol": {"bytes": 16.0 * n_c * n_c, "flops": n_c ** 3 / 3.0 + 2.0 * n_c ** 2},
        "backsub": {"bytes": obs + lm_back, "impl_bytes": obs + lm_back + pair + M * 9 * t,
                    "flops": 40.0 * N + 24.0 * P},
        "schur_blocks": blocks,
    }


def traffic_of(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu record, or None when the kernels' source
    changed since the counters were taken (or no record exists)."""
    import hashlib
    try:
        with open(TRAFFIC) as f:
            rec = json.load(f).get(kernel)
        with open(KERNEL_SOURCE, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_sha256") != sha or rec.get("workload") != workload:
        return None
    return rec.get("dram_bytes_per_launch")


def chol_kernel_name(ctx_mode_blocked: bool) -> str:
    return "k_blk_load + k_chol_cluster" if ctx_mode_blocked else "k_chol_cluster"


def roofline(prof: dict, wm: dict, workload: str, only_hbm: bool = False, chol_name: str = "k_chol_cluster") -> dict:
    """Achieved vs peak for each kernel with a work model, keyed by part name."""
    pk, pk_kind = peaks()
    out = {}
    for k, ms in prof.items():
        if k not in wm or ms <= 0:
            continue
        if k in ("chol", "schur_group"):
            if only_hbm:
                continue
            fp32 = wm[k].get("fp32", False)
            peak = FP32_NOMINAL_TFLOPS if fp32 else FP64_NOMINAL_GFLOPS / 1e3
            ach = wm[k]["flops"] / (ms * 1e-3) / 1e12
            out[k] = {"kernel": chol_name if k == "chol" else "k_schur_group", "bound": "alu", "achieved": ach,
                      "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                      "peak_source": ("FP32: 152 SMs x 128 lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s" if fp32 else
                                      "FP64: GB300 nominal 1.25 TFLOP/s (a probe measured 1.19)") +
                                     "; MEASURED_PEAKS.json has no FP32/FP64 figure",
                      "algorithmic_flops": wm[k]["flops"], "ms_per_launch": ms}
            if "impl_bytes" in wm[k]:
                out[k]["impl_gbs"] = wm[k]["impl_bytes"] / (ms * 1e-3) / 1e9
        else:
            ach = wm[k]["bytes"] / (ms * 1e-3) / 1e9
            out[k] = {"kernel": "k_" + k, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                      "frac": ach / pk["hbm_gbs"], "peak_source": pk_kind + " (copy bandwidth, burst)",
                      "algorithmic_bytes": wm[k]["bytes"], "impl_bytes": wm[k]["impl_bytes"],
                      "impl_frac": wm[k]["impl_bytes"] / (ms * 1e-3) / 1e9 / pk["hbm_gbs"], "ms_per_launch": ms}
        t = traffic_of(out[k]["kernel"], workload)
        out[k]["traffic"] = t
        if t is not None:
            out[k]["traffic_over_algorithmic"] = t / wm[k]["bytes"]
    return out


def load_golden(name: str):
    path = os.path.join(GOLDEN, f"{name}_oracle.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


# ---------------------------------------------------------------- small solves (f1-f4)

def small_solves(cvba, synth, dev, l2_flush, reps: int = 3):
    """Motion-only BA (multi-camera PnP), the loop-closure relative pose, multi-view
    triangulation and pose-graph optimisation: device time of each batched solve (CUDA
    events, L2 flushed before each repetition), its throughput, the roofline of its single
    kernel (algorithmic FLOPs per launch / time against the FP32 or FP64 rate), and its
    error against the oracle on a sample."""
    import torch
    from oracle import ba, pnp, pgo, relpose
    from oracle import triangulate as tri
    out = {}
    stream = torch.cuda.current_stream(dev)
    t = lambda a, dt=torch.float64: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    launches = 0

    def timed(fn):
        ms = []
        for k in range(reps + 1):
            l2_flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            stream.synchronize()
            if k > 0:
                ms.append(e0.elapsed_time(e1))
        return float(np.median(ms))

    def alu(flops, ms, fp32):
        peak = FP32_NOMINAL_TFLOPS if fp32 else FP64_NOMINAL_GFLOPS / 1e3
        ach = flops / (ms * 1e-3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "algorithmic_flops": flops, "ms_per_launch": ms,
                "peak_source": "FP32 152 x 128 x 2 x 2.07 GHz" if fp32 else "FP64 nominal 1.25 TFLOP/s"}

    # --- f1: motion-only BA, 512 frames of the 32-camera ring (~1.5M observations)
    b = synth.make_frames("pnp_multi")
    res = {"workload": "512 frames of the 16-pair ring, 400 map points each (%d observations), %d LM iterations"
                       % (b.N, b.iters)}
    per_obs = 250.0            # FLOPs per observation and iteration: linearisation ~200, candidate ~50
    for dtype, name in ((0, "fp64"), (1, "fp32")):
        ft = torch.float64 if dtype == 0 else torch.float32
        intr, tcb, pw, uv = t(b.rig.intr, ft), t(b.rig.T_cb.reshape(-1, 12), ft), t(b.lm, ft), t(b.obs_uv, ft)
        off, cm, lmi = t(b.frame_off, torch.int32), t(b.obs_cam, torch.int32), t(b.obs_lm, torch.int32)
        p0 = t(b.poses0.reshape(b.F, 12))
        poses = p0.clone()

        def run():
            poses.copy_(p0)
            cvba.cvba_pnp_solve(dtype, b.F, b.C, b.M, b.N, intr.data_ptr(), tcb.data_ptr(), pw.data_ptr(),
                                off.data_ptr(), cm.data_ptr(), lmi.data_ptr(), uv.data_ptr(), poses.data_ptr(),
                                b.iters, b.huber_delta, stream=stream.cuda_stream)
        ms = timed(run)
        launches += (reps + 1) * 2
        P = poses.cpu().numpy().reshape(b.F, 3, 4)
        sample = list(range(0, b.F, 32))
        t0 = time.perf_counter()
        ref = pnp.solve_frames(b, frames=sample)
        t_or = time.perf_counter() - t0
        err = pose_errors(P[sample], np.stack([T for T, _ in ref]))
        res[name] = {"value": b.F / (ms * 1e-3), "unit": "frames/s", "gobs_per_s": b.N * b.iters / (ms * 1e-3) / 1e9,
                     "ms": ms, "roofline": alu(per_obs * b.N * b.iters, ms, dtype == 1),
                     "vs_oracle": dict(err, frames=len(sample)), "oracle_frames_per_s": len(sample) / t_or}
    out["pnp"] = res

    # --- f2: loop-closure relative pose, the same frames with a map pose each
    T_mw, T_bm0 = synth.make_map_poses(b, seed=1)
    intr, tcb, pw, uv = t(b.rig.intr), t(b.rig.T_cb.reshape(-1, 12)), t(b.lm), t(b.obs_uv)
    off, cm, lmi = t(b.frame_off, torch.int32), t(b.obs_cam, torch.int32), t(b.obs_lm, torch.int32)
    mw, bm0 = t(T_mw.reshape(b.F, 12)), t(T_bm0.reshape(b.F, 12))
    bm = bm0.clone()

    def run_rel():
        bm.copy_(bm0)
        cvba.cvba_relpose_solve(0, b.F, b.C, b.M, b.N, intr.data_ptr(), tcb.data_ptr(), pw.data_ptr(), off.data_ptr(),
                                cm.data_ptr(), lmi.data_ptr(), uv.data_ptr(), mw.data_ptr(), bm.data_ptr(), b.iters,
                                b.huber_delta, stream=stream.cuda_stream)
    ms = timed(run_rel)
    launches += (reps + 1) * 2
    sample = list(range(0, b.F, 32))
    ref = relpose.solve_queries(b, T_mw, T_bm0, frames=sample)
    Tbm = bm.cpu().numpy().reshape(b.F, 3, 4)
    out["relpose"] = {"workload": "the same 512 frames, each against a map pose", "precision": "fp64",
                      "value": b.F / (ms * 1e-3), "unit": "queries/s", "ms": ms,
                      "roofline": alu(per_obs * b.N * b.iters, ms, False),
                      "vs_oracle": dict(pose_errors(Tbm[sample], np.stack([T for T, _ in ref])), frames=len(sample))}

    # --- f4: triangulation of the 200k landmarks of the 100-keyframe window (3.75M observations)
    q = synth.make_problem("c4", outlier_frac=0.0)
    order, loff = synth.landmark_segments(q.obs_lm, q.M)
    kf_s, cam_s, uv_s = q.obs_kf[order], q.obs_cam[order], q.obs_uv[order]
    res = {"workload": "200,000 landmarks of the 100-keyframe ring window from 3.75M observations, 10 LM iterations"}
    per_obs_t = 2 * 40.0 + 10 * 180.0    # linear step with refinement + per refinement iteration
    for dtype, name in ((0, "fp64"), (1, "fp32")):
        ft = torch.float64 if dtype == 0 else torch.float32
        intr, tcb, uvt = t(q.rig.intr, ft), t(q.rig.T_cb.reshape(-1, 12), ft), t(uv_s, ft)
        poses = t(q.poses_gt.reshape(q.K, 12))
        offt, kft, camt = t(loff, torch.int32), t(kf_s, torch.int32), t(cam_s, torch.int32)
        pwo = torch.zeros(q.M * 3, dtype=torch.float64, device=dev)

        def run_tri():
            cvba.cvba_triangulate(dtype, q.M, q.K, q.C, q.N, intr.data_ptr(), tcb.data_ptr(), poses.data_ptr(),
                                  offt.data_ptr(), kft.data_ptr(), camt.data_ptr(), uvt.data_ptr(), pwo.data_ptr(), 10,
                                  q.huber_delta, stream=stream.cuda_stream)
        ms = timed(run_tri)
        launches += reps + 1
        Pt = pwo.cpu().numpy().reshape(q.M, 3)
        sel = list(range(0, q.M, 400))
        ref = tri.triangulate(q.rig.intr, q.rig.T_cb, q.poses_gt, loff, kf_s, cam_s, uv_s, 10, q.huber_delta,
                              landmarks=sel)
        rel = [np.linalg.norm(Pt[j] - r[1]) / np.linalg.norm(r[1]) for j, r in zip(sel, ref) if r[2] == 0]
        res[name] = {"value": q.M / (ms * 1e-3), "unit": "landmarks/s", "ms": ms,
                     "gobs_per_s": q.N * 10 / (ms * 1e-3) / 1e9,
                     "roofline": alu(per_obs_t * q.N, ms, dtype == 1),
                     "vs_oracle": {"max_rel_point_error": float(max(rel)), "landmarks": len(rel)}}
    out["triangulation"] = res

    # --- f3: pose-graph optimisation, the 600-keyframe four-lap map
    g = synth.make_pose_graph("pgo_large")
    ed, de, p0 = t(g.edges, torch.int32), t(g.deltas.reshape(g.E, 12)), t(g.poses0.reshape(g.K, 12))
    pos = p0.clone()
    need = cvba.cvba_pgo_workspace_bytes(g.K, g.E)
    work = torch.empty(need, dtype=torch.uint8, device=dev)

    def run_pgo():
        pos.copy_(p0)
        cvba.cvba_pgo_solve(g.K, g.E, ed.data_ptr(), de.data_ptr(), pos.data_ptr(), g.iters, g.fixed,
                            work=work.data_ptr(), work_bytes=need, stream=stream.cuda_stream)
    ms = timed(run_pgo)
    n = 6 * (g.K - 1)
    npan = (n + 31) // 32
    launches += (reps + 1) * (2 + g.iters * (8 + 3 * npan))
    # work of the factorisation over the factor's profile (each row from the column of its
    # pose's first coupled pose): per 32-column panel the diagonal factor, the solve of the
    # rows below inside the envelope and their trailing update
    col = np.where(np.arange(g.K) == g.fixed, -1, np.cumsum(np.arange(g.K) != g.fixed) - 1)
    first = np.arange(g.K - 1)
    for i, j in np.asarray(g.edges).reshape(-1, 2):
        a, b = col[i], col[j]
        if a >= 0 and b >= 0:
            hi_, lo_ = max(a, b), min(a, b)
            first[hi_] = min(first[hi_], lo_)
    row_first = 6 * first[np.arange(n) // 6]
    fac_flops = 0.0
    for pn in range(npan):
        rows = np.nonzero(row_first[32 * (pn + 1):] <= 32 * pn + 31)[0]
        below = 0 if rows.size == 0 else ((32 * (pn + 1) + rows[-1] + 1 + 31) // 32 * 32 - 32 * (pn + 1))
        fac_flops += 32.0 ** 3 / 3.0 + below * 32.0 ** 2 + below * below * 32.0
    Po, _, _, otr = pgo.lm_solve(g.poses0, g.edges, g.deltas, g.iters, fixed=g.fixed)
    out["pgo"] = {"workload": "600 keyframes on four laps, %d edges, %d LM iterations" % (g.E, g.iters),
                  "precision": "fp64", "value": g.iters / (ms * 1e-3), "unit": "LM iters/s", "ms": ms,
                  "roofline": alu(g.iters * (fac_flops + 4.0 * n * n), ms, False),
                  "vs_oracle": pose_errors(pos.cpu().numpy().reshape(g.K, 3, 4), Po)}
    out["gpu_launches"] = launches
    return out


# ------------------------------------------------------------------------- reference

def oracle_sample(p, seconds: float, max_iters: int):
    """Oracle-S (block-sparse FP64 oracle, OpenMP on the host cores) run from the initial
    state for up to `max_iters` LM iterations or about `seconds` of CPU time; returns
    (iterations, elapsed seconds, threads)."""
    from oracle import ba, ba_sparse
    w = ba.Window.from_problem(p)
    sw = ba_sparse.SparseWindow(w)
    poses, lms, lam, nu = p.poses0.copy(), p.lm0.copy(), 1e-4, 2.0
    t0 = time.perf_counter()
    n_it = 0
    while n_it < max_iters:
        poses, lms, lam, nu, _ = ba_sparse.lm_iteration(sw, poses, lms, lam, nu)
        n_it += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    threads = sw.threads
    sw.close()
    return n_it, dt, threads


def run_reference(args):
    """The oracle (Oracle-S: exact block-sparse FP64 normal equations, on the host cores) on
    the same workload: each step is one LM iteration of its solve from the initial state
    (a bounded sample of the 15-iteration solve)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import ba, ba_sparse
    from paper_2506_04359_gb300 import synth
    p = synth.make_problem(args.workload)
    w = ba.Window.from_problem(p)
    sw = ba_sparse.SparseWindow(w)
    poses, lms, lam, nu = p.poses0.copy(), p.lm0.copy(), 1e-4, 2.0
    for _ in range(args.warmup):
        ba_sparse.lm_iteration(sw, poses, lms, lam, nu)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        poses, lms, lam, nu, _ = ba_sparse.lm_iteration(sw, poses, lms, lam, nu)
    dt = time.perf_counter() - t0
    v = args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "LM iters/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "K": p.K, "C": p.C, "M": p.M, "N": p.N, "precision": "fp64",
                   "step": "one LM iteration of the oracle (block-sparse FP64 normal equations, generic sparse "
                           "Cholesky, OpenMP)"},
        "cpu_baseline": {"value": v, "unit": "LM iters/s", "cores": sw.threads, "kind": "oracle",
                         "sample": f"LM iterations {args.warmup + 1}..{args.warmup + args.steps} of the "
                                   f"{args.workload} window"},
        "e2e": {"value": v, "unit": "LM iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    sw.close()


# ------------------------------------------------------------------------------- ours

def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2506_04359_gb300 import cvba, synth

    p = synth.make_problem(args.workload)
    precision = args.precision or ("mixed" if p.precision == "mixed" else "fp64")
    stream = torch.cuda.Stream(device=dev)
    l2_flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    extra_launches = 0

    def timed_solves(q, ctx, steps, warmup):
        """Device time of `steps` solves of window q from its initial state (reset on the
        device, inside the events), L2 flushed between solves outside the events."""
        q_p = torch.tensor(q.poses0.reshape(q.K, 12), dtype=torch.float64, device=dev)
        q_l = torch.tensor(q.lm0, dtype=torch.float64, device=dev)
        for _ in range(warmup):
            with torch.cuda.stream(stream):
                ctx.cvba_set_poses_dev(q_p.data_ptr())
                ctx.cvba_set_landmarks_dev(q_l.data_ptr())
                ctx.cvba_solve_async(q.iters, huber_delta=q.huber_delta)
        stream.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(steps):
                l2_flush.fill_(float(k))
                ev[k][0].record(stream)
                ctx.cvba_set_poses_dev(q_p.data_ptr())
                ctx.cvba_set_landmarks_dev(q_l.data_ptr())
                ctx.cvba_solve_async(q.iters, huber_delta=q.huber_delta)
                ev[k][1].record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        barrier(ws)
        wall = time.perf_counter() - t0
        dev_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
        launches = steps * (ctx.cvba_solve_launch_count(q.iters) + 2)
        return dev_s, wall, launches

    def vs_golden(q, gold, P, rms):
        if gold is None:
            return None
        return dict(pose_errors(P, np.array(gold["final_poses"])), rms_px=abs(rms - gold["final_rms_px"]))

    # --- main timed run (mixed by default)
    ctx = cvba.Context(precision, device=local, stream=stream.cuda_stream).load(p)
    sizes = ctx.cvba_get_sizes()
    P = sizes["P"]
    with ClockSampler(local) as cs:
        dev_s, wall, launches = timed_solves(p, ctx, args.steps, args.warmup)
    dev_s = max_over_ranks(dev_s, ws)
    tr = ctx.cvba_get_trace(p.iters)
    ev = ctx.cvba_evaluate(p.huber_delta)
    final_poses = ctx.cvba_get_poses()                 # before profiling moves the state on
    iters_total = args.steps * p.iters * ws
    value = iters_total / dev_s
    gobs = float(np.sum(tr["n_valid"])) * args.steps * ws / dev_s / 1e9
    gold = load_golden(args.workload)

    # --- roofline of every kernel with a work model (CUDA events around each kernel of one
    #     iteration, on the library's stream), and the dominant one
    prof = ctx.cvba_profile_iteration(10, huber_delta=p.huber_delta)
    wm = work_model(p, P, precision == "mixed")
    label = f"{args.workload} {precision}"
    blocked = 6 * (p.K - 1) >= 320
    roofs = roofline(prof, wm, label, chol_name=chol_kernel_name(blocked))
    dom = max(roofs, key=lambda k: roofs[k]["ms_per_launch"])
    roof = dict(roofs[dom])
    roof["workload"] = label
    roof["parts_ms"] = prof
    ctx.close()

    # --- FP64 path on the same window
    fp64 = None
    if precision != "fp64":
        c64 = cvba.Context("fp64", device=local, stream=stream.cuda_stream).load(p)
        n64 = max(3, args.steps // 4)
        d64, _, l64 = timed_solves(p, c64, n64, 1)
        extra_launches += l64
        d64 = max_over_ranks(d64, ws)
        rms64 = c64.cvba_evaluate(p.huber_delta)["rms"]
        fp64 = {"value": n64 * p.iters * ws / d64, "unit": "LM iters/s", "rms_px": rms64,
                "vs_oracle": vs_golden(p, gold, c64.cvba_get_poses(), rms64)}
        c64.close()

    # --- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        h_intr, h_tcb = pin(p.rig.intr), pin(p.rig.T_cb.reshape(-1, 12))
        h_wh = pin(p.rig.wh.astype(np.int32))
        h_poses, h_lms = pin(p.poses0.reshape(p.K, 12)), pin(p.lm0)
        h_kf, h_cam, h_lm = pin(p.obs_kf.astype(np.int32)), pin(p.obs_cam.astype(np.int32)), pin(p.obs_lm.astype(np.int32))
        h_uv = pin(p.obs_uv)
        out_p = pin(np.zeros((p.K, 3, 4)))
        out_l = pin(np.zeros((p.M, 3)))
        ce = cvba.Context(precision, device=local, stream=stream.cuda_stream)

        def e2e_step():
            ce.cvba_set_rig(h_intr, h_tcb, h_wh)
            ce.cvba_set_poses(h_poses, p.fixed_kf)
            ce.cvba_set_landmarks(h_lms)
            ce.cvba_set_observations(h_kf, h_cam, h_lm, h_uv)
            ce.cvba_solve(p.iters, huber_delta=p.huber_delta)
            cvba.lib.cvba_get_poses(ce._h, cvba._dptr(out_p))
            cvba.lib.cvba_get_landmarks(ce._h, cvba._dptr(out_l))

        n_e2e = max(3, args.steps // 4)
        for _ in range(min(args.warmup, 2)):
            e2e_step()
        barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        torch.cuda.synchronize()
        barrier(ws)
        e2e_s = max_over_ranks(time.perf_counter() - t0, ws)
        h2d = sum(a.nbytes for a in (h_intr, h_tcb, h_wh, h_poses, h_lms, h_kf, h_cam, h_lm, h_uv))
        d2h = out_p.nbytes + out_l.nbytes + p.iters * 64
        extra_launches += n_e2e * (ce.cvba_solve_launch_count(p.iters) + 2)
        e2e = {"value": n_e2e * p.iters * ws / e2e_s, "unit": "LM iters/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * e2e_s / n_e2e, "steps": n_e2e,
               "note": "each step: set rig, poses, landmarks, observations (host layout and upload), solve, "
                       "read poses and landmarks"}
        ce.close()

    # --- CPU baseline: Oracle-S on a bounded sample (rank 0, N = 1)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        n_it, dt, thr = oracle_sample(p, 12.0, p.iters)
        cpu = {"value": n_it / dt, "unit": "LM iters/s", "cores": thr, "kind": "oracle",
               "sample": f"first {n_it} LM iterations of the {args.workload} window (Oracle-S: block-sparse "
                         f"FP64 normal equations, generic sparse Cholesky, OpenMP)"}

    # --- extra sections: the 20-keyframe stereo window, and 256 batched windows
    c1 = None
    batched = None
    if not args.no_extras:
        q = synth.make_problem("c1") if args.workload != "c1" else p
        g1 = load_golden("c1")
        c1 = {"workload": "c1", "K": q.K, "C": q.C, "M": q.M, "N": q.N, "iters": q.iters}
        for prec in ("mixed", "fp64"):
            cq = cvba.Context(prec, device=local, stream=stream.cuda_stream).load(q)
            t_q, _, lq = timed_solves(q, cq, 10, 2)
            extra_launches += lq
            rq = cq.cvba_evaluate(q.huber_delta)["rms"]
            c1[prec] = {"value": 10 * q.iters / t_q, "unit": "LM iters/s", "rms_px": rq,
                        "vs_oracle": vs_golden(q, g1, cq.cvba_get_poses(), rq)}
            if prec == "mixed":
                pq = cq.cvba_profile_iteration(10, huber_delta=q.huber_delta)
                c1[prec]["parts_ms"] = pq
                c1[prec]["roofline"] = roofline(pq, work_model(q, cq.cvba_get_sizes()["P"], True), "c1 mixed")
            cq.close()

        wins = synth.make_batch(256)
        g3 = load_golden("c3")
        bctx = [cvba.Context("mixed", device=local, stream=stream.cuda_stream).load(w) for w in wins]
        batch = cvba.Batch(bctx)
        tuned = batch.cvba_batch_autotune(iters=2)
        for c, w in zip(bctx, wins):
            c.cvba_set_poses(w.poses0, w.fixed_kf)
            c.cvba_set_landmarks(w.lm0)
        it_b = wins[0].iters
        batch.cvba_batch_solve(it_b)                       # warm-up (captures the graph)
        n_steps = 3
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_steps)]
        for k in range(n_steps):
            for c, w in zip(bctx, wins):                   # host resets, outside the events
                c.cvba_set_poses(w.poses0, w.fixed_kf)
                c.cvba_set_landmarks(w.lm0)
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                l2_flush.fill_(float(k))
                evs[k][0].record(stream)
                batch.cvba_batch_solve_async(it_b)
                evs[k][1].record(stream)
            stream.synchronize()
        t_b = sum(a.elapsed_time(b) for a, b in evs) / 1e3
        extra_launches += n_steps * batch.cvba_batch_launch_count(it_b)
        gate = None
        if g3 is not None:
            diffs = [abs(c.cvba_evaluate(w.huber_delta)["rms"] - g["final_rms_px"])
                     for c, w, g in zip(bctx, wins, g3["windows"])]
            gate = {"max_rms_diff_px": float(max(diffs)), "windows_within_1e-3_px": int(sum(d <= 1e-3 for d in diffs)),
                    "n_windows": len(diffs)}
        n_obs_b = sum(w.N for w in wins)
        seq = {}
        for prec in ("fp64", "mixed"):
            cs_ = [cvba.Context(prec, device=local, stream=stream.cuda_stream).load(w) for w in wins]
            for c in cs_:
                c.cvba_solve_async(it_b)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                for c in cs_:
                    c.cvba_solve_async(it_b)
                e1.record(stream)
            stream.synchronize()
            seq[prec] = len(wins) * it_b / (e0.elapsed_time(e1) / 1e3)
            extra_launches += sum(c.cvba_solve_launch_count(it_b) for c in cs_)
            for c in cs_:
                c.close()
        batched = {"workload": "c3 (256 windows, K 5-30, M 300-3000, 1/2/4/8 stereo pairs)", "precision": "mixed",
                   "iters": it_b, "value": n_steps * len(wins) * it_b / t_b, "unit": "window LM iters/s",
                   "gobs_per_s": n_obs_b * it_b * n_steps / t_b / 1e9, "ms_per_solve": 1e3 * t_b / n_steps,
                   "one_by_one_fp64": seq["fp64"], "one_by_one_mixed": seq["mixed"], "autotuned": tuned,
                   "vs_oracle": gate}
        batch.close()
        for c in bctx:
            c.close()

    small = None
    if not args.no_extras:
        small = small_solves(cvba, synth, dev, l2_flush)
        extra_launches += small.pop("gpu_launches")

    golden_rms = gold["final_rms_px"] if gold else None
    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "LM iters/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "K": p.K, "C": p.C, "M": p.M, "N": p.N, "pairs": P,
                       "precision": precision, "lm_iters_per_step": p.iters, "parallelism": "replicas",
                       "l2": "flushed between steps (512 MiB write outside the timed events)"},
            "gobs_per_s": gobs,
            "rms_px": ev["rms"], "rms_oracle_px": golden_rms,
            "rms_ok": None if golden_rms is None else bool(abs(ev["rms"] - golden_rms) <= 1e-3),
            "vs_oracle": vs_golden(p, gold, final_poses, ev["rms"]),
            "fp64": fp64,
            "roofline": roof,
            "roofline_all": roofs,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": cs.summary(),
            "c1": c1,
            "batched": batched,
            "small_solves": small,
            "gpu_launches": launches,
            "gpu_launches_extras": extra_launches,
            "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
