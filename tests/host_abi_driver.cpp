// Test driver (CPU only): the C ABI's argument checks, call order and checkpoint format, run
// through cvba_host.cpp over the CUDA runtime stand-in of cuda_standin.h (no kernel runs, so
// only what the host layer decides is exercised).  It loads the window written by
// test_host_abi.py, makes a fixed sequence of calls and writes "<name> <status>" per call.
//
//   host_abi_driver <dir>
//     reads   <dir>/ (the window files of host_tables_driver)
//     writes  <dir>/status.txt
#include <cstdlib>
#include <fstream>
#include <limits>

#include "cvba_host.cpp"
#include "cuda_standin.h"

namespace {
template <typename T>
std::vector<T> read_vec(const std::string& path, size_t n) {
  std::vector<T> v(n);
  std::ifstream(path, std::ios::binary).read(reinterpret_cast<char*>(v.data()), (std::streamsize)(n * sizeof(T)));
  return v;
}
}  // namespace

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  const std::string d = argv[1];
  std::ofstream out(d + "/status.txt");
  auto rec = [&](const char* name, cvba_status s, const cvba_ctx* c = nullptr) {
    out << name << " " << (int)s;
    if (c && s != CVBA_OK) out << " " << cvba_last_error(c);
    out << "\n";
  };
  int K = 0, C = 0, M = 0, N = 0, fixed = 0;
  std::ifstream(d + "/dims.txt") >> K >> C >> M >> N >> fixed;
  const auto kf = read_vec<int32_t>(d + "/kf.bin", N), cam = read_vec<int32_t>(d + "/cam.bin", N);
  const auto lm = read_vec<int32_t>(d + "/lm.bin", N);
  const auto uv = read_vec<double>(d + "/uv.bin", 2 * (size_t)N), intr = read_vec<double>(d + "/intr.bin", 4 * (size_t)C);
  const auto tcb = read_vec<double>(d + "/tcb.bin", 12 * (size_t)C), poses = read_vec<double>(d + "/poses.bin", 12 * (size_t)K);
  const auto lms = read_vec<double>(d + "/lms.bin", 3 * (size_t)M);
  const double nan = std::nan("");
  cvba_opts o{};
  o.iters = 2;
  o.huber_delta = 1.0;
  o.lambda0 = 1e-4;
  o.z_min = 0.05;
  o.reset_lambda = 1;
  o.refine = -1;

  cvba_ctx* bad = nullptr;
  rec("create_bad_precision", cvba_create(&bad, 0, nullptr, (cvba_precision)7));
  rec("create_bad_device", cvba_create(&bad, 3, nullptr, CVBA_FP64));
  cvba_ctx* c = nullptr;
  rec("create", cvba_create(&c, 0, nullptr, CVBA_FP64));
  rec("solve_before_setters", cvba_solve(c, &o, nullptr), c);
  rec("observations_before_setters", cvba_set_observations(c, N, kf.data(), cam.data(), lm.data(), uv.data()), c);
  {
    size_t b0 = 0;
    rec("get_state_before_layout", cvba_get_state(c, nullptr, &b0), c);
  }
  rec("get_layout_before_layout", cvba_get_layout(c, nullptr, nullptr, nullptr), c);
  // rig
  rec("rig_zero_cameras", cvba_set_rig(c, 0, intr.data(), tcb.data(), nullptr), c);
  rec("rig_65_cameras", cvba_set_rig(c, 65, intr.data(), tcb.data(), nullptr), c);
  {
    auto in2 = intr;
    in2[1] = nan;
    rec("rig_nonfinite", cvba_set_rig(c, C, in2.data(), tcb.data(), nullptr), c);
    std::vector<int32_t> wh((size_t)C * 2, 640);
    wh[1] = 0;
    rec("rig_zero_image_size", cvba_set_rig(c, C, intr.data(), tcb.data(), wh.data()), c);
  }
  rec("rig", cvba_set_rig(c, C, intr.data(), tcb.data(), nullptr), c);
  // poses
  rec("poses_one_keyframe", cvba_set_poses(c, 1, poses.data(), 0), c);
  rec("poses_257_keyframes", cvba_set_poses(c, 257, poses.data(), 0), c);
  rec("poses_fixed_out_of_range", cvba_set_poses(c, K, poses.data(), K), c);
  {
    auto p2 = poses;
    p2[5] = nan;
    rec("poses_nonfinite", cvba_set_poses(c, K, p2.data(), fixed), c);
  }
  rec("poses", cvba_set_poses(c, K, poses.data(), fixed), c);
  // landmarks
  rec("landmarks_none", cvba_set_landmarks(c, 0, lms.data()), c);
  {
    auto l2 = lms;
    l2[4] = nan;
    rec("landmarks_nonfinite", cvba_set_landmarks(c, M, l2.data()), c);
  }
  {
    // a large array (checked over several threads): one non-finite value near the end
    cvba_ctx* big = nullptr;
    cvba_create(&big, 0, nullptr, CVBA_FP64);
    std::vector<double> many((size_t)3 * 50000, 1.0);
    rec("landmarks_many", cvba_set_landmarks(big, 50000, many.data()), big);
    many[many.size() - 2] = std::numeric_limits<double>::infinity();
    rec("landmarks_many_nonfinite", cvba_set_landmarks(big, 50000, many.data()), big);
    cvba_destroy(big);
  }
  rec("landmarks", cvba_set_landmarks(c, M, lms.data()), c);
  // observations
  {
    auto cam2 = cam;
    cam2[3] = C + 5;
    rec("observations_camera_out_of_range", cvba_set_observations(c, N, kf.data(), cam2.data(), lm.data(), uv.data()), c);
    auto lm2 = lm;
    lm2[N - 1] = -1;
    rec("observations_landmark_negative", cvba_set_observations(c, N, kf.data(), cam.data(), lm2.data(), uv.data()), c);
    auto kf2 = kf;
    kf2[0] = K;
    rec("observations_keyframe_out_of_range", cvba_set_observations(c, N, kf2.data(), cam.data(), lm.data(), uv.data()), c);
    auto uv2 = uv;
    uv2[3] = nan;
    rec("observations_nonfinite", cvba_set_observations(c, N, kf.data(), cam.data(), lm.data(), uv2.data()), c);
    // landmark 0 left with one observation
    std::vector<int32_t> k3, c3, l3;
    std::vector<double> u3;
    bool kept = false;
    for (int n = 0; n < N; ++n) {
      if (lm[n] == 0) {
        if (kept) continue;
        kept = true;
      }
      k3.push_back(kf[n]), c3.push_back(cam[n]), l3.push_back(lm[n]), u3.push_back(uv[2 * n]), u3.push_back(uv[2 * n + 1]);
    }
    rec("observations_single_view_landmark",
        cvba_set_observations(c, (int)k3.size(), k3.data(), c3.data(), l3.data(), u3.data()), c);
  }
  rec("observations_none", cvba_set_observations(c, 0, kf.data(), cam.data(), lm.data(), uv.data()), c);
  rec("observations", cvba_set_observations(c, N, kf.data(), cam.data(), lm.data(), uv.data()), c);
  // options and settings
  {
    cvba_opts b = o;
    b.huber_delta = -1.0;
    rec("solve_negative_huber", cvba_solve(c, &b, nullptr), c);
    b = o;
    b.refine = 9;
    rec("solve_refine_9", cvba_solve(c, &b, nullptr), c);
    b = o;
    b.iters = -1;
    rec("solve_negative_iters", cvba_solve(c, &b, nullptr), c);
    b = o;
    b.z_min = nan;
    rec("solve_nonfinite_zmin", cvba_solve(c, &b, nullptr), c);
  }
  // the captured solve graph: kept while the options and the device view are unchanged
  // (new state values change neither), rebuilt when either changes
  {
    const int g0 = g_instantiate_count;
    cvba_solve(c, &o, nullptr);
    cvba_solve(c, &o, nullptr);
    out << "graphs_same " << g_instantiate_count - g0 << "\n";
    cvba_opts o3 = o;
    o3.iters = 3;
    cvba_solve(c, &o3, nullptr);
    out << "graphs_iters " << g_instantiate_count - g0 << "\n";
    cvba_set_landmarks(c, M, lms.data());
    cvba_set_poses(c, K, poses.data(), fixed);
    cvba_solve(c, &o3, nullptr);
    out << "graphs_new_state " << g_instantiate_count - g0 << "\n";
    cvba_set_observations(c, N, kf.data(), cam.data(), lm.data(), uv.data());
    cvba_solve(c, &o3, nullptr);
    out << "graphs_same_window_again " << g_instantiate_count - g0 << "\n";
    cvba_set_tuning(c, 32, 8);                     // the sizes the window had already: same view
    cvba_solve(c, &o3, nullptr);
    out << "graphs_same_tuning " << g_instantiate_count - g0 << "\n";
    cvba_set_tuning(c, 64, 16);
    cvba_solve(c, &o3, nullptr);
    out << "graphs_tuning " << g_instantiate_count - g0 << "\n";
    rec("chol_mode_2", cvba_set_chol_mode(c, 2), c);
    rec("solve_blocked", cvba_solve(c, &o3, nullptr), c);
    out << "graphs_chol_mode " << g_instantiate_count - g0 << "\n";
    cvba_set_tuning(c, 0, 0);
    cvba_set_chol_mode(c, 0);
  }
  rec("chol_mode_3", cvba_set_chol_mode(c, 3), c);
  rec("tuning_negative", cvba_set_tuning(c, -1, 0), c);
  rec("damping_set", cvba_set_damping(c, 0.5, 3.0), c);
  // checkpoint: size query, round trip into a fresh context, refusals
  size_t bytes = 0;
  rec("state_size", cvba_get_state(c, nullptr, &bytes), c);
  std::vector<unsigned char> state(bytes);
  size_t got = bytes;
  rec("state_get", cvba_get_state(c, state.data(), &got), c);
  out << "state_bytes " << bytes << " " << got << "\n";
  cvba_ctx* e = nullptr;
  cvba_create(&e, 0, nullptr, CVBA_FP64);
  cvba_set_rig(e, C, intr.data(), tcb.data(), nullptr);
  {
    auto p2 = poses;
    for (int a = 0; a < K; ++a) p2[a * 12 + 3] += 1.0;           // another state of the same problem
    auto l2 = lms;
    for (auto& x : l2) x *= 1.5;
    cvba_set_poses(e, K, p2.data(), fixed);
    cvba_set_landmarks(e, M, l2.data());
  }
  cvba_set_observations(e, N, kf.data(), cam.data(), lm.data(), uv.data());
  rec("state_truncated", cvba_set_state(e, state.data(), bytes - 8), e);
  {
    auto garbage = state;
    for (size_t i = 0; i < 16 && i < garbage.size(); ++i) garbage[i] ^= 0x5a;
    rec("state_garbage", cvba_set_state(e, garbage.data(), bytes), e);
  }
  rec("state_set", cvba_set_state(e, state.data(), bytes), e);
  {
    std::vector<double> pa((size_t)K * 12), pb((size_t)K * 12), la((size_t)M * 3), lb((size_t)M * 3);
    cvba_get_poses(c, pa.data());
    cvba_get_poses(e, pb.data());
    cvba_get_landmarks(c, la.data());
    cvba_get_landmarks(e, lb.data());
    double lam = 0, nu = 0;
    cvba_get_damping(e, &lam, &nu);
    out << "state_restored " << (pa == pb && la == lb && pa == poses && la == lms ? 1 : 0) << " " << lam << " " << nu
        << "\n";
  }
  {
    // a context holding another problem (one landmark fewer) refuses the checkpoint
    cvba_ctx* f = nullptr;
    cvba_create(&f, 0, nullptr, CVBA_FP64);
    cvba_set_rig(f, C, intr.data(), tcb.data(), nullptr);
    cvba_set_poses(f, K, poses.data(), fixed);
    cvba_set_landmarks(f, M - 1, lms.data());
    std::vector<int32_t> k4, c4, l4;
    std::vector<double> u4;
    for (int n = 0; n < N; ++n)
      if (lm[n] != M - 1)
        k4.push_back(kf[n]), c4.push_back(cam[n]), l4.push_back(lm[n]), u4.push_back(uv[2 * n]), u4.push_back(uv[2 * n + 1]);
    rec("other_problem_layout", cvba_set_observations(f, (int)k4.size(), k4.data(), c4.data(), l4.data(), u4.data()), f);
    rec("state_other_problem", cvba_set_state(f, state.data(), bytes), f);
    cvba_destroy(f);
  }
  cvba_destroy(e);
  cvba_destroy(c);
  out << "done 0\n";
  return 0;
}
