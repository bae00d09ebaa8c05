// Test driver (CPU only): the batched solve's host logic (cvba_host.cpp over the CUDA runtime
// stand-in of cuda_standin.h, with cvba_layout.cpp linked beside it) on windows written by
// test_host_batch.py.  It writes what a test needs to check the batch plan (the per-window
// views and the (window, item) work lists of every phase), when the captured graph is rebuilt,
// the refusal of a window without a layout, and the autotuner under scripted timings (the
// candidate it picks, the tuning it leaves on every window, the state it restores, its cache).
//
//   host_batch_driver <dir> <fp64|mixed> <n_windows>
//     reads   <dir>/w<i>/ (the window files of host_tables_driver), <dir>/timings.txt (elapsed
//             times in the order the autotuner reads them; two scripts of 24, one per run)
//     writes  <dir>/out.txt (name value... lines), <dir>/lists_<tag>.bin (the work lists)
#include <cstdlib>
#include <fstream>

#include "cvba_host.cpp"
#include "cuda_standin.h"

namespace {
template <typename T>
std::vector<T> read_vec(const std::string& path, size_t n) {
  std::vector<T> v(n);
  std::ifstream(path, std::ios::binary).read(reinterpret_cast<char*>(v.data()), (std::streamsize)(n * sizeof(T)));
  return v;
}
void need(bool ok, const char* what) {
  if (!ok) {
    std::fprintf(stderr, "failed: %s\n", what);
    std::exit(3);
  }
}
cvba_ctx* load(const std::string& d, cvba_precision prec) {
  int K = 0, C = 0, M = 0, N = 0, fixed = 0;
  std::ifstream(d + "/dims.txt") >> K >> C >> M >> N >> fixed;
  const auto kf = read_vec<int32_t>(d + "/kf.bin", N), cam = read_vec<int32_t>(d + "/cam.bin", N);
  const auto lm = read_vec<int32_t>(d + "/lm.bin", N);
  const auto uv = read_vec<double>(d + "/uv.bin", 2 * (size_t)N), intr = read_vec<double>(d + "/intr.bin", 4 * (size_t)C);
  const auto tcb = read_vec<double>(d + "/tcb.bin", 12 * (size_t)C), poses = read_vec<double>(d + "/poses.bin", 12 * (size_t)K);
  const auto lms = read_vec<double>(d + "/lms.bin", 3 * (size_t)M);
  cvba_ctx* c = nullptr;
  need(cvba_create(&c, 0, nullptr, prec) == CVBA_OK, "create");
  need(cvba_set_rig(c, C, intr.data(), tcb.data(), nullptr) == CVBA_OK, "rig");
  need(cvba_set_poses(c, K, poses.data(), fixed) == CVBA_OK, "poses");
  need(cvba_set_landmarks(c, M, lms.data()) == CVBA_OK, "landmarks");
  need(cvba_set_observations(c, N, kf.data(), cam.data(), lm.data(), uv.data()) == CVBA_OK, "observations");
  return c;
}
}  // namespace

int main(int argc, char** argv) {
  if (argc < 4) return 2;
  const std::string dir = argv[1];
  const cvba_precision prec = std::string(argv[2]) == "mixed" ? CVBA_MIXED : CVBA_FP64;
  const int n = std::atoi(argv[3]);
  std::ofstream out(dir + "/out.txt");
  std::vector<cvba_ctx*> ctx;
  for (int i = 0; i < n; ++i) ctx.push_back(load(dir + "/w" + std::to_string(i), prec));
  cvba_opts o{};
  o.iters = 3;
  o.huber_delta = 1.0;
  o.lambda0 = 1e-4;
  o.z_min = 0.05;
  o.reset_lambda = 1;
  o.refine = -1;

  // a window without a layout is refused
  {
    cvba_ctx* bare = nullptr;
    need(cvba_create(&bare, 0, nullptr, prec) == CVBA_OK, "create bare");
    std::vector<cvba_ctx*> with_bare = ctx;
    with_bare.push_back(bare);
    cvba_batch* bb = nullptr;
    need(cvba_batch_create(&bb, n + 1, with_bare.data()) == CVBA_OK, "batch with bare");
    out << "bare_status " << (int)cvba_batch_solve_async(bb, &o) << "\n";
    cvba_batch_destroy(bb);
    cvba_destroy(bare);
  }

  cvba_batch* b = nullptr;
  need(cvba_batch_create(&b, n, ctx.data()) == CVBA_OK, "batch");
  // the plan: views and work lists, written as (tag, window, item) triples
  auto dump = [&](const std::string& tag) {
    const BatchLaunch& L = b->L;
    std::vector<int32_t> v;
    auto add = [&](int id, const int2* items, int cnt) {
      for (int i = 0; i < cnt; ++i) {
        v.push_back(id);
        v.push_back(items[i].x);
        v.push_back(items[i].y);
      }
    };
    add(0, L.lin_items, L.n_lin);
    add(1, L.kf_items, L.n_kf);
    add(2, L.schur_items, L.n_schur);
    add(3, L.blk_items, L.n_blkit);
    add(4, L.direct_items, L.n_direct);
    add(5, L.win_items, n);
    std::ofstream(dir + "/lists_" + tag + ".bin", std::ios::binary)
        .write(reinterpret_cast<const char*>(v.data()), (std::streamsize)(v.size() * 4));
    int views_equal = 1;
    for (int w = 0; w < n; ++w)
      views_equal &= std::memcmp(&L.wins[w], &ctx[w]->d, sizeof(Dev)) == 0 ? 1 : 0;
    const size_t lists_at = reinterpret_cast<const char*>(L.lin_items) - static_cast<const char*>(b->dbuf);
    out << "views_equal_" << tag << " " << views_equal << "\n";
    out << "lists_aligned_" << tag << " " << (lists_at % 16 == 0 && lists_at >= sizeof(Dev) * n ? 1 : 0) << "\n";
    out << "chol_cs_" << tag << " " << L.chol_cs << "\n";
    for (int w = 0; w < n; ++w)
      out << "tiles_" << tag << "_" << w << " " << ctx[w]->d.n_lin_tiles << " " << ctx[w]->K << " "
          << ctx[w]->d.n_schur_tiles << " " << ctx[w]->act_blk.size() << " " << ctx[w]->d.n_direct_tiles << "\n";
  };
  need(cvba_batch_solve_async(b, &o) == CVBA_OK, "solve 1");
  dump("first");
  out << "graphs_after_first " << g_instantiate_count << "\n";
  need(cvba_batch_solve_async(b, &o) == CVBA_OK, "solve 2");
  out << "graphs_after_same " << g_instantiate_count << "\n";
  o.iters = 4;
  need(cvba_batch_solve_async(b, &o) == CVBA_OK, "solve 3");
  out << "graphs_after_iters " << g_instantiate_count << "\n";
  need(cvba_set_tuning(ctx[n - 1], 32, 8) == CVBA_OK, "tuning");
  need(cvba_batch_solve_async(b, &o) == CVBA_OK, "solve 4");
  out << "graphs_after_tuning " << g_instantiate_count << "\n";
  dump("tuned");
  need(cvba_batch_set_chol_cluster(b, 8) == CVBA_OK, "cluster");
  need(cvba_batch_solve_async(b, &o) == CVBA_OK, "solve 5");
  out << "graphs_after_cluster " << g_instantiate_count << "\n";
  dump("cluster");

  // autotuner: scripted timings; the state of every window is restored
  std::vector<float> script;
  {
    std::ifstream t(dir + "/timings.txt");
    for (float x; t >> x;) script.push_back(x);
  }
  need(script.size() == 48, "two scripts of 24 timings");
  auto state = [&](int w) {
    std::vector<double> s((size_t)ctx[w]->K * 12 + (size_t)ctx[w]->M * 3);
    need(cvba_get_poses(ctx[w], s.data()) == CVBA_OK, "get poses");
    need(cvba_get_landmarks(ctx[w], s.data() + (size_t)ctx[w]->K * 12) == CVBA_OK, "get landmarks");
    return s;
  };
  std::vector<std::vector<double>> before;
  for (int w = 0; w < n; ++w) before.push_back(state(w));
  for (int run = 0; run < 3; ++run) {
    if (run == 2) cvba_batch_autotune_clear();
    g_elapsed_script.assign(script.begin() + (run == 2 ? 24 : 0), script.begin() + (run == 2 ? 48 : 24));
    g_elapsed_calls = 0;
    int bl = 0, bs = 0, bc = 0;
    need(cvba_batch_autotune(b, &o, &bl, &bs, &bc) == CVBA_OK, "autotune");
    int restored = 1, applied = 1;
    for (int w = 0; w < n; ++w) {
      restored &= state(w) == before[w] ? 1 : 0;
      applied &= ctx[w]->tune_lin_pairs == bl && ctx[w]->tune_schur_lms == bs ? 1 : 0;
    }
    out << "autotune_" << run << " " << bl << " " << bs << " " << bc << " " << g_elapsed_calls << " " << restored
        << " " << applied << " " << b->chol_cs << "\n";
  }
  cvba_batch_destroy(b);
  for (cvba_ctx* c : ctx) cvba_destroy(c);
  out << "done 1\n";
  return 0;
}
