// Test driver (CPU only): the library's host layer (cvba_host.cpp, compiled into this file,
// with cvba_layout.cpp linked beside it) over the CUDA runtime stand-in of cuda_standin.h, in
// which device memory is host memory, copies are memcpy, streams, events and graphs are tokens
// and the kernel launchers do nothing.  Fresh "device" memory is filled with 0xCD bytes, so a
// buffer that the layout should zero and does not shows up.  It loads a window through the C
// ABI and writes what the layout hands to the kernels, so that test_host_tables.py can check
// every table against its definition without a GPU.  Built and run by test_host_tables.py.
//
//   host_tables_driver <dir> <fp64|mixed> <lin_tile_pairs> <schur_tile_landmarks> <chol_mode>
//     reads   dims.txt (K C M N fixed_kf), kf.bin cam.bin lm.bin (int32 N), uv.bin (f64 2N),
//             intr.bin (f64 4C), tcb.bin (f64 12C), poses.bin (f64 12K), lms.bin (f64 3M),
//             poses2.bin, lms2.bin (replacements set after the layout)
//     writes  one file per table, t_<name>.bin, and t_sizes.txt
#include <cstdlib>
#include <fstream>

#include "cvba_host.cpp"
#include "cuda_standin.h"

// ---------------------------------------------------------------- driver
namespace {
std::string g_dir;

template <typename T>
std::vector<T> read_vec(const std::string& name, size_t n) {
  std::vector<T> v(n);
  std::ifstream(g_dir + "/" + name, std::ios::binary).read(reinterpret_cast<char*>(v.data()), (std::streamsize)(n * sizeof(T)));
  return v;
}
template <typename T>
void put(const std::string& name, const T* p, size_t n) {
  std::ofstream(g_dir + "/t_" + name + ".bin", std::ios::binary)
      .write(reinterpret_cast<const char*>(p), (std::streamsize)(n * sizeof(T)));
}
int check(cvba_status s, cvba_ctx* c, const char* what) {
  if (s != CVBA_OK) {
    std::fprintf(stderr, "%s: status %d: %s\n", what, (int)s, c ? cvba_last_error(c) : "");
    std::exit(3);
  }
  return 0;
}
}  // namespace

int main(int argc, char** argv) {
  if (argc < 6) return 2;
  g_dir = argv[1];
  const bool mixed = std::string(argv[2]) == "mixed";
  const int lin_pairs = std::atoi(argv[3]), schur_lms = std::atoi(argv[4]), chol_mode = std::atoi(argv[5]);
  int K = 0, C = 0, M = 0, N = 0, fixed = 0;
  {
    std::ifstream d(g_dir + "/dims.txt");
    d >> K >> C >> M >> N >> fixed;
  }
  const auto kf = read_vec<int32_t>("kf.bin", N), cam = read_vec<int32_t>("cam.bin", N), lm = read_vec<int32_t>("lm.bin", N);
  const auto uv = read_vec<double>("uv.bin", 2 * (size_t)N), intr = read_vec<double>("intr.bin", 4 * (size_t)C);
  const auto tcb = read_vec<double>("tcb.bin", 12 * (size_t)C), poses = read_vec<double>("poses.bin", 12 * (size_t)K);
  const auto lms = read_vec<double>("lms.bin", 3 * (size_t)M);
  const auto poses2 = read_vec<double>("poses2.bin", 12 * (size_t)K), lms2 = read_vec<double>("lms2.bin", 3 * (size_t)M);

  cvba_ctx* c = nullptr;
  check(cvba_create(&c, 0, nullptr, mixed ? CVBA_MIXED : CVBA_FP64), nullptr, "create");
  check(cvba_set_chol_mode(c, chol_mode), c, "chol mode");
  check(cvba_set_rig(c, C, intr.data(), tcb.data(), nullptr), c, "rig");
  check(cvba_set_poses(c, K, poses.data(), fixed), c, "poses");
  check(cvba_set_landmarks(c, M, lms.data()), c, "landmarks");
  check(cvba_set_observations(c, N, kf.data(), cam.data(), lm.data(), uv.data()), c, "observations");
  if (lin_pairs > 0 || schur_lms > 0) check(cvba_set_tuning(c, lin_pairs, schur_lms), c, "tuning");
  // a second load of the same window into the same context: buffers and staging are reused
  check(cvba_set_observations(c, N, kf.data(), cam.data(), lm.data(), uv.data()), c, "observations again");

  const Dev& d = c->d;
  const int P = d.P, n_c = d.n_c;
  put("lm_order", c->lm_order.data(), M);
  put("obs_order", c->obs_order.data(), N);
  put("d_lm_order", c->d_lm_order, M);
  if (mixed)
    put("obs_uv", static_cast<const float*>(d.obs_uv), 2 * (size_t)N);
  else
    put("obs_uv", static_cast<const double*>(d.obs_uv), 2 * (size_t)N);
  put("obs_cam", d.obs_cam, N);
  put("pair_kf", d.pair_kf, P);
  put("pair_lm", d.pair_lm, P);
  put("pair_obs", d.pair_obs, (size_t)P + 1);
  put("lm_pair", d.lm_pair, (size_t)M + 1);
  put("lm_blk", d.lm_blk, (size_t)M + 1);
  put("kf_pb", d.kf_pb, K);
  std::vector<int32_t> lt, st, dt;
  for (int i = 0; i < d.n_lin_tiles; ++i) {
    const LinTile& t = d.lin_tiles[i];
    for (int v : {t.l0, t.l1, t.p0, t.p1, t.kf_lo, t.kf_n, t.part_off, t.kfl_off, t.o0, t.o1, t.kfi0, t.kfi_n}) lt.push_back(v);
  }
  auto schur = [](std::vector<int32_t>& out, const SchurTile* p, int n) {
    for (int i = 0; i < n; ++i) {
      const SchurTile& t = p[i];
      for (int v : {t.l0, t.l1, t.p0, t.p1, t.b0, t.b1, t.k_lo, t.span, t.direct, t.part_off}) out.push_back(v);
    }
  };
  schur(st, d.schur_tiles, d.n_schur_tiles);
  schur(dt, d.direct_tiles, d.n_direct_tiles);
  put("lin_tiles", lt.data(), lt.size());
  put("schur_tiles", st.data(), st.size());
  put("direct_tiles", dt.data(), dt.size());
  size_t kfl = 0, kfi = 0;
  for (int i = 0; i < d.n_lin_tiles; ++i) {
    kfl = std::max(kfl, (size_t)d.lin_tiles[i].kfl_off + d.lin_tiles[i].kf_n + 1);
    kfi = std::max(kfi, (size_t)d.lin_tiles[i].kfi0 + d.lin_tiles[i].kfi_n);
  }
  put("lin_kf_off", d.lin_kf_off, kfl);
  put("lin_kf_slot", d.lin_kf_slot, kfl);
  put("lin_kf_idx", d.lin_kf_idx, kfi);
  put("kf_tiles_off", d.kf_tiles_off, (size_t)K + 1);
  put("blk_tiles_off", d.blk_tiles_off, (size_t)d.n_blk + 1);
  int32_t n_bt = 0;
  std::memcpy(&n_bt, d.blk_tiles_off + d.n_blk, 4);
  put("blk_part_at", d.blk_part_at, (size_t)n_bt);
  put("act_blk", d.act_blk, (size_t)d.n_act);
  put("panel_end", d.panel_end, (size_t)kMaxPanels);
  put("rig", d.rig, (size_t)C * RIG_STRIDE);
  put("pose0", d.pose[0], (size_t)K * POSE_STRIDE);
  put("lm0", d.lm[0], (size_t)M * 3);
  if (mixed) {
    put("rig_f", d.rig_f, (size_t)C * RIG_STRIDE);
    put("pose_f0", d.pose_f[0], (size_t)K * POSE_STRIDE);
    put("lm_f0", d.lm_f[0], (size_t)M * 3);
  }
  put("S", d.S, (size_t)n_c * n_c);
  put("dc", d.dc, (size_t)n_c);
  put("dp", d.dp, (size_t)M * 3);
  put("lin_part", d.lin_part, (size_t)d.n_lin_tiles * 4);
  put("bs_part", d.bs_part, (size_t)d.n_lin_tiles * 8);
  {
    const double ctl[3] = {(double)d.ctrl->cur, d.ctrl->lam, d.ctrl->nu};
    put("ctrl", ctl, 3);
  }
  // replaced state after the layout: only that half is written, into the current buffer
  check(cvba_set_landmarks(c, M, lms2.data()), c, "landmarks after layout");
  put("lm0_after_lms", d.lm[0], (size_t)M * 3);
  put("pose0_after_lms", d.pose[0], (size_t)K * POSE_STRIDE);
  if (mixed) put("lm_f0_after_lms", d.lm_f[0], (size_t)M * 3);
  check(cvba_set_poses(c, K, poses2.data(), fixed), c, "poses after layout");
  put("pose0_after_poses", d.pose[0], (size_t)K * POSE_STRIDE);
  if (mixed) put("pose_f0_after_poses", d.pose_f[0], (size_t)K * POSE_STRIDE);
  std::vector<double> got_l((size_t)M * 3), got_p((size_t)K * 12);
  check(cvba_get_landmarks(c, got_l.data()), c, "get landmarks");
  check(cvba_get_poses(c, got_p.data()), c, "get poses");
  put("got_lms", got_l.data(), got_l.size());
  put("got_poses", got_p.data(), got_p.size());
  {
    std::ofstream s(g_dir + "/t_sizes.txt");
    s << P << " " << n_c << " " << d.n_blk << " " << d.npw << " " << d.chol_blocked << " " << d.max_span << " "
      << kMaxPanels << " " << LIN_TILE_PAIRS << " " << LIN_TILE_LMS << " " << SCHUR_TILE_PAIRS << " "
      << SCHUR_TILE_LMS << " " << SPAN_MAX << " " << RIG_STRIDE << " " << POSE_STRIDE << "\n";
  }
  cvba_destroy(c);
  return 0;
}
