// Test driver (CPU only): runs the library's host layout (cvba_layout.cpp) on observations
// read from binary files and writes every array it produces, and exercises the host worker
// pool with nested and concurrent parallel sections.  Built and run by test_host_layout.py.
//
//   host_layout_driver layout <dir>   reads dims.txt (K C M N fixed), kf.bin, cam.bin, lm.bin
//                                     (int32); writes out.bin (lm_order, lm_rank, obs_order,
//                                     lm_off, obs_cam, pair_kf, pair_lm, pair_obs, lm_pair) and
//                                     sizes.txt (P), or err.txt if the layout is rejected
//   host_layout_driver pool           nested and concurrent sections, and ranges over few
//                                     large items; exit status 0 if every task ran exactly once
#include <atomic>
#include <cstdio>
#include <fstream>
#include <string>
#include <thread>
#include <vector>

#include "cvba_internal.h"

using namespace cvba;

static std::vector<int32_t> read_i32(const std::string& path, size_t n) {
  std::vector<int32_t> v(n);
  std::ifstream(path, std::ios::binary).read(reinterpret_cast<char*>(v.data()), (std::streamsize)(n * 4));
  return v;
}

static int run_layout(const std::string& dir) {
  int K = 0, C = 0, M = 0, N = 0, fixed = 0;
  {
    std::ifstream d(dir + "/dims.txt");
    d >> K >> C >> M >> N >> fixed;
  }
  const auto kf = read_i32(dir + "/kf.bin", N), cam = read_i32(dir + "/cam.bin", N), lm = read_i32(dir + "/lm.bin", N);
  HostLayout L;
  std::string err;
  if (!compute_host_layout(K, C, M, N, fixed, kf.data(), cam.data(), lm.data(), L, err)) {
    std::ofstream(dir + "/err.txt") << err;
    return 0;
  }
  // a second call on the same work arrays must give the same layout
  HostLayout L2;
  compute_host_layout(K, C, M, N, fixed, kf.data(), cam.data(), lm.data(), L2, err);
  compute_host_layout(K, C, M, N, fixed, kf.data(), cam.data(), lm.data(), L2, err);
  if (L2.obs_order != L.obs_order || L2.pair_obs != L.pair_obs) return 3;
  std::ofstream o(dir + "/out.bin", std::ios::binary);
  for (const auto* v : {&L.lm_order, &L.lm_rank, &L.obs_order, &L.lm_off, &L.obs_cam, &L.pair_kf, &L.pair_lm,
                        &L.pair_obs, &L.lm_pair})
    o.write(reinterpret_cast<const char*>(v->data()), (std::streamsize)(v->size() * 4));
  std::ofstream(dir + "/sizes.txt") << L.pair_kf.size();
  return 0;
}

static int run_pool() {
  std::atomic<long> sum{0};
  for (int rep = 0; rep < 100; ++rep)
    parallel_tasks(8, [&](int t) {
      parallel_tasks(4, [&](int u) { sum += t * 10 + u; });              // nested section
      parallel_for(10000, 4, [&](int64_t a, int64_t b, int) { sum += b - a; });
    });
  long want = 100L * (8 * 10000 + 4 * (0 + 10 + 20 + 30 + 40 + 50 + 60 + 70) + 8 * (0 + 1 + 2 + 3));
  std::vector<std::thread> callers;                                       // concurrent sections
  for (int c = 0; c < 4; ++c)
    callers.emplace_back([&] {
      for (int rep = 0; rep < 100; ++rep) parallel_for(100000, 8, [&](int64_t a, int64_t b, int) { sum += b - a; });
    });
  for (auto& th : callers) th.join();
  want += 4L * 100 * 100000;
  for (int64_t n : {0, 1, 3, 300, 100000}) {                              // every item exactly once
    std::vector<std::atomic<int>> seen((size_t)n);
    parallel_ranges(n, [&](int64_t a, int64_t b, int) {
      for (int64_t i = a; i < b; ++i) seen[i]++;
    });
    for (auto& s : seen) sum += s.load();
    want += n;
  }
  std::printf("%ld %ld\n", sum.load(), want);
  return sum.load() == want ? 0 : 1;
}

int main(int argc, char** argv) {
  if (argc >= 3 && std::string(argv[1]) == "layout") return run_layout(argv[2]);
  if (argc >= 2 && std::string(argv[1]) == "pool") return run_pool();
  return 2;
}
